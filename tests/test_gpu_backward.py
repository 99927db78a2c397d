"""GPU adjoint (dgs_render_backward through the C ABI) against the FP64 oracle's adjoint.

L = sum(g_C * RGB) + sum(g_D * D) with seeded upstream gradients that are zero at every pixel
the oracle marks ambiguous (an FP32 renderer may take the other branch there; those pixels are
checked branch by branch by the forward tests) or where a contributor's gradient switch -- the
alpha clamp, the Jacobian guard, the colour clamp at 0 -- lies within its FP32 band (the
rendered value is continuous there but its derivative is not).

Tolerance per gradient tensor: |g - g*| <= 1e-3 |g*| + 1e-5 max|g*| for every entry but at most a
1e-5 fraction of them, those few within ten times that bound, and a relative L2 error of at most
1e-4.  The outliers are thin, nearly opaque splats whose gradient is a sum of large per-pixel
terms: an FP32 projected centre (error ~1e-4 px) moves it by (Hessian x 1e-4), which exceeds the
element bound while the tensor stays accurate.
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


def _gradients(sc, seed=0, mode="batched", dtype="f32", oracle_scene=None):
    """GPU gradients of `sc` stored as `dtype`, and the oracle's for `oracle_scene` (default sc)
    under the same upstream gradients."""
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    osc = sc if oracle_scene is None else oracle_scene
    ds = DeviceScene(sc, device="cuda:0", dtype=dtype)
    r = Renderer(mode=mode)
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
    ref = O.backward_scene(osc, gCv, gDv, O.OracleOptions())
    r.close()
    return node_grads, gposes, ref


def _check(name, g, r):
    g = np.asarray(g, np.float64)
    scale = np.abs(r).max()
    err = np.abs(g - r)
    tol = RTOL * np.abs(r) + ATOL_FRAC * scale
    bad = err > tol
    info = (name, int(bad.sum()), bad.size, float(err.max()), float(scale))
    assert bad.sum() <= int(1e-5 * bad.size), info
    assert np.all(err <= 10 * tol), info
    assert np.linalg.norm(g - r) <= 1e-4 * max(np.linalg.norm(r), 1e-30), info


def _compare(sc, node_grads, gposes, ref):
    off = 0
    for k, nd in enumerate(sc.nodes):
        sl = slice(off, off + nd.n)
        off += nd.n
        nc = (nd.sh_degree + 1) ** 2
        G = {n: t.cpu().numpy() for n, t in node_grads[k].items()}
        _check(f"node{k}.mean", G["mean"], ref["mean"][sl])
        _check(f"node{k}.log_scale", G["log_scale"], ref["log_scale"][sl])
        _check(f"node{k}.quat", G["quat"], ref["quat"][sl])
        _check(f"node{k}.opacity_logit", G["opacity_logit"], ref["opacity_logit"][sl])
        _check(f"node{k}.sh", G["sh"], ref["sh"][sl, :nc])
    _check("poses", gposes.cpu().numpy(), ref["pose"])


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
