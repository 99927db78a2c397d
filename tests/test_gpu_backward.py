"""GPU adjoint (dgs_render_backward through the C ABI) against the FP64 oracle's adjoint.

L = sum(g_C * RGB) + sum(g_D * D) with seeded upstream gradients that are zero at every pixel
the oracle marks ambiguous (an FP32 renderer may take the other branch there; those pixels are
checked branch by branch by the forward tests) or where a contributor's gradient switch -- the
alpha clamp, the Jacobian guard, the colour clamp at 0 -- lies within its FP32 band (the
rendered value is continuous there but its derivative is not).

Tolerance per gradient entry (no figure in the paper or the method's statement):
|g - g*| <= 1e-3 |g*| + 1e-5 max|g*| + 2 e*, and per tensor a relative L2 error of at most 1e-4.
e* is the oracle's FP32 error model of that entry (header of oracle_backward_view): every
composited (pixel, Gaussian) pair contributes absolute error bounds of its per-instance partials
(alpha and transmittance rounding, the cancellation in (C_out - P_i) / T_{i+1}, colour, depth and
centre rounding, the FP32 accumulation over the pixels), carried through the chain rule in
absolute value.  It matters where an entry is a small residue of large per-pixel terms of both
signs (thin, nearly opaque splats), for which a bound relative to the entry itself is too tight.
"""

import numpy as np
import pytest

import oracle as O
from paper_2507_21981_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL, ATOL_FRAC = 1e-3, 1e-5


def _with_sh(sc, deg, seed):
    rng = np.random.default_rng(seed)
    nodes = []
    for nd in sc.nodes:
        sh = rng.normal(0, 0.2, (nd.n, (deg + 1) ** 2, 3)).astype(np.float32)
        sh[:, 0] = nd.sh[:, 0]
        nodes.append(S.GaussianNode(nd.mean, nd.log_scale, nd.quat, nd.opacity_logit, sh, deg, nd.name))
    sc.nodes = nodes
    return sc


def _gradients(sc, seed=0, mode="batched", dtype="f32", oracle_scene=None, **ropts):
    """GPU gradients of `sc` stored as `dtype`, and the oracle's (with its FP32 error model) for
    `oracle_scene` (default sc) under the same upstream gradients; ropts are Renderer options."""
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    osc = sc if oracle_scene is None else oracle_scene
    ds = DeviceScene(sc, device="cuda:0", dtype=dtype)
    r = Renderer(mode=mode, **ropts)
    rgb, depth, _ = r.render(ds)
    rng = np.random.default_rng(seed)
    pk = O.oracle._Packed(osc)
    gC = np.zeros((ds.n_pixels, 3), np.float32)
    gD = np.zeros(ds.n_pixels, np.float32)
    gCv, gDv = [], []
    for v, (e, c) in enumerate(sc.views):
        ref = O.render_view(osc, e, c, O.OracleOptions(), pk)
        H, W = ref.depth.shape
        amb = (ref.n_alt > 0) | (ref.tol_rgb > 0) | ref.grad_amb
        g = rng.normal(size=(H, W, 3)).astype(np.float32)
        d = (rng.normal(size=(H, W)) * 0.3).astype(np.float32)
        g[amb] = 0
        d[amb] = 0
        sl = ds.view_slice(v)
        gC[sl] = g.reshape(-1, 3)
        gD[sl] = d.reshape(-1)
        gCv.append(g.astype(np.float64))
        gDv.append(d.astype(np.float64))
    node_grads, gposes = r.backward(ds, rgb, depth, torch.from_numpy(gC).cuda(), torch.from_numpy(gD).cuda())
    torch.cuda.synchronize()
    ref = O.backward_scene(osc, gCv, gDv, O.OracleOptions(), with_error=True)
    r.close()
    return node_grads, gposes, ref


def _check(name, g, r, e, counts=None):
    """Every entry within the bound; counts[name] = entries that needed the error-model term."""
    g = np.asarray(g, np.float64)
    scale = np.abs(r).max()
    err = np.abs(g - r)
    r18 = RTOL * np.abs(r) + ATOL_FRAC * scale
    tol = r18 + 2 * e
    bad = np.argwhere(err > tol)
    info = (name, len(bad), g.size, float(err.max()), float(scale),
            [(tuple(int(x) for x in i), float(g[tuple(i)]), float(r[tuple(i)]), float(e[tuple(i)])) for i in bad[:3]])
    assert len(bad) == 0, info
    assert np.linalg.norm(g - r) <= 1e-4 * max(np.linalg.norm(r), 1e-30), info
    if counts is not None:
        counts[name] = int((err > r18).sum())


def _compare(sc, node_grads, gposes, ref, counts=None):
    off = 0
    for k, nd in enumerate(sc.nodes):
        sl = slice(off, off + nd.n)
        nc = (nd.sh_degree + 1) ** 2
        G = {n: t.cpu().numpy() for n, t in node_grads[k].items()}
        for name in ("mean", "log_scale", "quat", "opacity_logit", "sh"):
            r, e = ref[name][sl], ref["err_" + name][sl]
            if name == "sh":
                r, e = r[:, :nc], e[:, :nc]
            _check(f"node{k}.{name}", G[name], r, e, counts)
        off += nd.n
    _check("poses", gposes.cpu().numpy(), ref["pose"], ref["err_pose"], counts)


def test_backward_fd_subset_sh3():
    sc = _with_sh(S.fd_subset(seed=2), 3, seed=2)
    _compare(sc, *_gradients(sc, seed=2))


def test_backward_config1_plain_and_batched_agree_with_oracle():
    sc = S.config1(seed=3)
    for mode in ("batched", "plain"):
        _compare(sc, *_gradients(sc, seed=3, mode=mode))


def test_backward_room_and_posed_objects():
    sc = S.config4(seed=2, n_bg=30_000, n_obj=2_000, res=160, f=140.0)
    _compare(sc, *_gradients(sc, seed=4))


def test_backward_many_views_share_the_background():
    sc = S.config2(seed=5, n_envs=3, n_bg=20_000, n_obj=1_000, width=96, height=72, f=75.0)
    _compare(sc, *_gradients(sc, seed=5))


def test_autograd_function_matches_direct_backward():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer, render_differentiable
    sc = _with_sh(S.config1(seed=6, n_bg=1500, n_obj=500, res=64, f=55.0), 2, seed=6)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer()
    params = ds.param_list()
    for p in params:
        p.requires_grad_(True)
    poses = ds.node_poses.clone().requires_grad_(True)
    rgb, depth, _ = render_differentiable(r, ds, poses)
    gen = torch.Generator(device="cuda").manual_seed(0)
    wC = torch.randn(rgb.shape, device="cuda", generator=gen)
    wD = torch.randn(depth.shape, device="cuda", generator=gen)
    ((rgb * wC).sum() + (depth * wD).sum()).backward()
    direct, gposes = r.backward(ds, rgb.detach(), depth.detach(), wC, wD)
    for k in range(len(sc.nodes)):
        for j, name in enumerate(ds.PARAM_NAMES):
            p = params[k * len(ds.PARAM_NAMES) + j]
            torch.testing.assert_close(p.grad, direct[k][name], rtol=1e-4, atol=1e-6)
    torch.testing.assert_close(poses.grad.reshape(gposes.shape), gposes, rtol=1e-4, atol=1e-6)
    r.close()


def test_backward_full_500k_view():
    """The differentiation workload: one 800x800 view of 500k SH-3 Gaussians and 8 posed nodes."""
    sc = S.config4(seed=1)
    _compare(sc, *_gradients(sc, seed=7))
