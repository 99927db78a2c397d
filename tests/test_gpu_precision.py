"""Reduced-precision attribute storage: log-scales, quaternions and SH coefficients in BF16 or
FP16, everything else FP32.

Compute error: the GPU render of the BF16/FP16 scene must match, pixel by pixel and branch by
branch, the FP64 oracle fed the same rounded attributes.  Storage error: the same render against
the oracle fed the FP32 attributes, reported as max-abs and PSNR = 10 log10(1/MSE) over RGB.
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_21981_gb300 import scenes as S
from tests.parity import compare_view

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_TDT = {"bf16": "bfloat16", "f16": "float16"}


def _rounded(sc, dtype):
    """The scene with log-scales, quaternions and SH rounded to `dtype` (and back to FP32)."""
    tdt = getattr(torch, _TDT[dtype])
    rd = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(tdt).float().numpy()
    nodes = [S.GaussianNode(nd.mean, rd(nd.log_scale), rd(nd.quat), nd.opacity_logit, rd(nd.sh), nd.sh_degree, nd.name)
             for nd in sc.nodes]
    return S.Scene(sc.name, nodes, sc.env_node_ids, sc.node_poses, sc.cams_per_env, sc.cam_intr, sc.cam_res,
                   sc.cam_pose, sc.meta)


def _render(sc, dtype):
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    ds = DeviceScene(sc, device="cuda:0", dtype=dtype)
    r = Renderer()
    out = [t.cpu().numpy() for t in r.render(ds)]
    r.close()
    return ds, out


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_low_precision_storage(dtype):
    sc = S.config2(seed=7, n_envs=2, n_bg=60_000, n_obj=3_000, width=160, height=120, f=125.0)
    ds, (rgb, depth, alpha) = _render(sc, dtype)
    rs = _rounded(sc, dtype)
    pk_r, pk_f = O.oracle._Packed(rs), O.oracle._Packed(sc)
    worst_psnr = np.inf
    for v, (e, c) in enumerate(sc.views):
        sl = ds.view_slice(v)
        ref = O.render_view(rs, e, c, O.OracleOptions(), pk_r)
        H, W = ref.depth.shape
        bad, rep = compare_view(rgb[sl].reshape(H, W, 3), depth[sl].reshape(H, W), ref, alpha[sl].reshape(H, W))
        assert bad == 0, rep                           # compute error: same tolerance as FP32
        full = O.render_view(sc, e, c, O.OracleOptions(), pk_f)
        mse = float(np.mean((rgb[sl].reshape(H, W, 3) - full.rgb) ** 2))
        worst_psnr = min(worst_psnr, 10 * np.log10(1.0 / max(mse, 1e-30)))
    # storage error against FP32 attributes (reported; a loose sanity floor)
    assert worst_psnr > 25.0, worst_psnr
    print(f"{dtype}: worst storage PSNR over {sc.n_views} views = {worst_psnr:.1f} dB")


def test_low_precision_backward_matches_oracle_on_rounded_attributes():
    from tests.test_gpu_backward import _compare, _gradients
    sc = S.config4(seed=3, n_bg=20_000, n_obj=1_500, res=128, f=112.0)
    rs = _rounded(sc, "bf16")
    # the GPU reads BF16 storage of sc; the oracle sees the same rounded values (rs)
    _compare(rs, *_gradients(sc, seed=8, dtype="bf16", oracle_scene=rs))


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_config5_full_size_sampled_views(dtype):
    """The precision-and-scale workload at full size (3M-Gaussian room + 6 x 50k objects,
    128 envs x 3 cameras, nodes in Z-order, graph replay): four seeded sampled views against
    the oracle fed the same rounded attributes (compute error, FP32 tolerance) and against the
    oracle fed FP32 attributes (storage error: max-abs and PSNR, reported)."""
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config5(seed=1)
    ds = DeviceScene(sc, device="cuda:0", dtype=dtype, spatial_order=True)
    r = Renderer(mode="graph")
    for _ in range(2):
        out = [t.cpu().numpy() for t in r.render(ds)]
    assert r.stats()["path"] == 1
    r.close()
    rgb, depth, alpha = out
    osc = ds.scene
    rs = _rounded(osc, dtype)
    pk_r, pk_f = O.oracle._Packed(rs), O.oracle._Packed(osc)
    views = sorted(int(v) for v in np.random.default_rng(11).choice(sc.n_views, 4, replace=False))
    lines = []
    for v in views:
        e, c = sc.views[v]
        sl = ds.view_slice(v)
        ref = O.render_view(rs, e, c, O.OracleOptions(), pk_r)
        H, W = ref.depth.shape
        img = rgb[sl].reshape(H, W, 3)
        bad, rep = compare_view(img, depth[sl].reshape(H, W), ref, alpha[sl].reshape(H, W))
        assert bad == 0, rep
        full = O.render_view(osc, e, c, O.OracleOptions(), pk_f)
        err = np.abs(img - full.rgb)
        psnr = 10 * np.log10(1.0 / max(float(np.mean(err ** 2)), 1e-30))
        lines.append(f"view {v}: max-abs {err.max():.4f} PSNR {psnr:.1f} dB")
        assert psnr > 25.0, lines[-1]
    print(f"config 5 {dtype} storage error vs FP32 attributes: " + "; ".join(lines))
