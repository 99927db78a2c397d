"""Depth -> TSDF fusion on the GPU (dgs_tsdf_integrate) against the FP64 oracle.

On every voxel whose decisions the oracle does not flag as FP32-ambiguous (a projection within
1e-3 px of a pixel edge, z near 0, sdf near -trunc): the weight W exactly, the field F within
1e-4.  Bound: the FP32 projection and the normalisation D / A carry a relative error of a few
u = 2^-24 on magnitudes below 3 m, i.e. 8u (|d| + |z| + |p| + |t| + 1) / trunc < 2e-5 per view
for trunc >= 0.04 m, plus the rounding of the running average (2 ulp per update with the
approximate reciprocal); 1e-4 covers both.  Cases: a sphere from 12 views, noisy partial-coverage
depth with gaps between views and a weight cap, sequential calls, and a 32^3 block of a 256^3 grid
fused from 64 views of 640 x 480.
"""
import numpy as np
import pytest

from oracle import tsdf as T
from paper_2507_21981_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL_F = 1e-4


def _gpu(F, W, origin, vox, trunc, wmax, amin, cams, depth_flat, alpha_flat, offs=None, r=None):
    from paper_2507_21981_gb300 import dgs as D
    from paper_2507_21981_gb300.render import Renderer
    own = r is None
    r = r or Renderer()
    dF, dW = torch.as_tensor(np.ascontiguousarray(F, np.float32)).cuda(), torch.as_tensor(np.ascontiguousarray(W, np.float32)).cuda()
    nz, ny, nx = F.shape
    rc = D.dgs_tsdf_integrate(r.ctx, dF, dW, nx, ny, nz, origin, vox, trunc, wmax, amin, D.cameras(cams), len(cams),
                              torch.as_tensor(depth_flat).cuda(), torch.as_tensor(alpha_flat).cuda(), offs,
                              torch.cuda.current_stream().cuda_stream)
    assert rc == D.DGS_OK, D.dgs_last_error(r.ctx)
    out = dF.cpu().numpy(), dW.cpu().numpy()
    if own:
        r.close()
    return out


def _check(gF, gW, rF, rW, amb, min_seen=1000):
    ok = ~amb
    assert (gW[ok] == rW[ok]).all(), int((gW[ok] != rW[ok]).sum())
    err = np.abs(gF[ok] - rF[ok])
    assert err.max() <= TOL_F, float(err.max())
    assert (rW[ok] > 0).sum() >= min_seen
    return float(err.max()), float(amb.mean())


def test_sphere_twelve_views():
    c = np.array([0.1, -0.2, 0.3])
    cams, Dv, Av = S.sphere_depth_views(c, 0.2, n_views=12, width=128, height=96, f=110.0, dist=1.0)
    n, vox = 48, 0.5 / 48
    origin = (c - 0.25).astype(np.float32)
    F0, W0 = np.zeros((n, n, n)), np.zeros((n, n, n))
    gF, gW = _gpu(F0, W0, origin, vox, 0.04, 100.0, 0.5, cams, Dv.reshape(-1), Av.reshape(-1))
    rF, rW, amb = T.integrate(F0, W0, origin.astype(np.float64), np.float32(vox), np.float32(0.04), 100.0, 0.5, cams,
                              Dv, Av)
    _check(gF, gW, rF, rW, amb)


def test_noisy_partial_coverage_gaps_cap_and_sequential_calls():
    c = np.array([0.0, 0.0, 0.0])
    cams, Dv, Av = S.sphere_depth_views(c, 0.25, n_views=10, width=80, height=64, f=70.0, dist=0.9, seed=3)
    rng = np.random.default_rng(4)
    A = np.clip(rng.uniform(0.2, 1.0, Av.shape), 0, 1).astype(np.float32) * Av
    D = (Dv * (1 + rng.normal(0, 0.01, Dv.shape))).astype(np.float32) * A          # unnormalised, noisy
    # views with gaps between them in the flat arrays
    offs, at = [], 0
    for _ in range(len(cams)):
        offs.append(at)
        at += 80 * 64 + 37
    Df = np.zeros(at, np.float32)
    Af = np.zeros(at, np.float32)
    for k, o in enumerate(offs):
        Df[o:o + 80 * 64] = D[k].reshape(-1)
        Af[o:o + 80 * 64] = A[k].reshape(-1)
    n, vox = 40, 0.6 / 40
    origin = np.array([-0.3, -0.3, -0.3], np.float32)
    F0, W0 = np.zeros((n, n, n)), np.zeros((n, n, n))
    from paper_2507_21981_gb300.render import Renderer
    r = Renderer()
    half = len(cams) // 2
    gF, gW = _gpu(F0, W0, origin, vox, 0.05, 4.0, 0.5, cams[:half], Df, Af, np.asarray(offs[:half], np.int64), r=r)
    gF, gW = _gpu(gF, gW, origin, vox, 0.05, 4.0, 0.5, cams[half:], Df, Af, np.asarray(offs[half:], np.int64), r=r)
    r.close()
    rF, rW, amb = T.integrate(F0, W0, origin.astype(np.float64), np.float32(vox), np.float32(0.05), 4.0, 0.5, cams, D, A)
    _check(gF, gW, rF, rW, amb)
    assert gW.max() == 4.0


def test_full_grid_block_sampled():
    """A 256^3 grid over a 0.8 m cube fused from 64 views of 640 x 480; the oracle recomputes a
    32^3 block in the middle of the grid (where the surface passes)."""
    c = np.array([0.0, 0.0, 0.0])
    cams, Dv, Av = S.sphere_depth_views(c, 0.3, n_views=64, width=640, height=480, f=500.0, dist=1.2, seed=9)
    n, vox = 256, 0.8 / 256
    origin = np.array([-0.4, -0.4, -0.4], np.float32)
    F0 = np.zeros((n, n, n), np.float32)
    gF, gW = _gpu(F0, F0, origin, vox, 0.02, 100.0, 0.5, cams, Dv.reshape(-1), Av.reshape(-1))
    assert np.isfinite(gF).all() and (gF <= 1).all() and gW.max() <= 64
    off = np.array([96, 128, 208])                # (k, j, i) corner of the block: near x = +0.25 m
    blk = (slice(off[0], off[0] + 32), slice(off[1], off[1] + 32), slice(off[2], off[2] + 32))
    o_blk = origin.astype(np.float64) + off[::-1] * np.float64(np.float32(vox))
    rF, rW, amb = T.integrate(np.zeros((32, 32, 32)), np.zeros((32, 32, 32)), o_blk, np.float32(vox), np.float32(0.02),
                              100.0, 0.5, cams, Dv, Av)
    # the block's voxel centres differ from the grid's by the rounding of the shifted origin
    _check(gF[blk], gW[blk], rF, rW, amb, min_seen=500)


def test_sphere_grid_whose_rows_are_not_a_multiple_of_four():
    """Rows of nx = 47 voxels take the one-voxel-per-thread kernel (the four-voxel kernel needs
    nx a multiple of 4); both must match the oracle."""
    c = np.array([0.05, 0.1, -0.1])
    cams, Dv, Av = S.sphere_depth_views(c, 0.2, n_views=8, width=96, height=80, f=90.0, dist=1.0, seed=7)
    nz, ny, nx, vox = 40, 44, 47, 0.5 / 46
    origin = (c - 0.25).astype(np.float32)
    F0, W0 = np.zeros((nz, ny, nx)), np.zeros((nz, ny, nx))
    gF, gW = _gpu(F0, W0, origin, vox, 0.04, 100.0, 0.5, cams, Dv.reshape(-1), Av.reshape(-1))
    rF, rW, amb = T.integrate(F0, W0, origin.astype(np.float64), np.float32(vox), np.float32(0.04), 100.0, 0.5, cams,
                              Dv, Av)
    _check(gF, gW, rF, rW, amb, min_seen=500)
