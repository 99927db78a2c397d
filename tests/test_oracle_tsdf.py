"""Pins of the TSDF fusion oracle (oracle/tsdf.py) against facts that do not come from it: a
head-on plane in closed form (projective distance, truncation, frustum), the normalisation of
the renderer's unnormalised depth by its coverage, the running average over views and the
weight cap, a sphere seen from many views whose fused field changes sign at the sphere's
radius, and single voxels placed exactly on the thresholds of the fusion's integer decisions.
No GPU is needed.
"""
import numpy as np

from oracle import tsdf as T
from paper_2507_21981_gb300 import scenes as S

CAM = (40.0, 40.0, 16.0, 16.0, 32, 32, np.eye(3, 4))     # at the origin looking along +z


def _vol(shape=(24, 8, 8)):
    return np.zeros(shape), np.zeros(shape)


def test_head_on_plane_closed_form():
    z0, mu, vox = 1.0, 0.05, 0.01
    origin = [-0.04, -0.04, 0.9]
    F, W = _vol()
    D = np.full((32, 32), z0)
    A = np.ones((32, 32))
    F, W, amb = T.integrate(F, W, origin, vox, mu, 100.0, 0.5, [CAM], [D], [A])
    z = origin[2] + (np.arange(24) + 0.5) * vox
    want_w = (z0 - z >= -mu).astype(float)
    want_f = np.where(want_w > 0, np.minimum(1.0, (z0 - z) / mu), 0.0)
    np.testing.assert_allclose(W[:, 4, 4], want_w)
    np.testing.assert_allclose(F[:, 4, 4], want_f, atol=1e-12)
    assert W[:, 0, 0].tolist() == W[:, 7, 7].tolist()      # the whole 8 cm slab is in view


def test_unnormalised_depth_and_coverage_threshold():
    origin, vox, mu = [-0.04, -0.04, 0.9], 0.01, 0.05
    ref = T.integrate(*_vol(), origin, vox, mu, 100.0, 0.5, [CAM], [np.full((32, 32), 1.0)], [np.ones((32, 32))])
    part = T.integrate(*_vol(), origin, vox, mu, 100.0, 0.5, [CAM], [np.full((32, 32), 0.6)], [np.full((32, 32), 0.6)])
    np.testing.assert_allclose(part[0], ref[0], atol=1e-12)
    low = T.integrate(*_vol(), origin, vox, mu, 100.0, 0.5, [CAM], [np.full((32, 32), 0.4)], [np.full((32, 32), 0.4)])
    assert (low[1] == 0).all()


def test_two_views_average_and_weight_cap():
    origin, vox, mu = [-0.04, -0.04, 0.9], 0.01, 0.05
    D1, D2, A = np.full((32, 32), 1.0), np.full((32, 32), 1.02), np.ones((32, 32))
    F, W, _ = T.integrate(*_vol(), origin, vox, mu, 100.0, 0.5, [CAM, CAM], [D1, D2], [A, A])
    z = origin[2] + (np.arange(24) + 0.5) * vox
    f1 = np.minimum(1, (1.0 - z) / mu)
    f2 = np.minimum(1, (1.02 - z) / mu)
    both = (1.0 - z >= -mu)
    np.testing.assert_allclose(F[both, 4, 4], (f1[both] + f2[both]) / 2, atol=1e-12)
    Fc, Wc, _ = T.integrate(*_vol(), origin, vox, mu, 1.0, 0.5, [CAM, CAM], [D1, D2], [A, A])
    assert Wc.max() == 1.0
    np.testing.assert_allclose(Fc[both, 4, 4], (f1[both] + f2[both]) / 2, atol=1e-12)


def test_sphere_zero_crossing():
    c, R = np.array([0.1, -0.2, 0.3]), 0.2
    cams, D, A = S.sphere_depth_views(c, R, n_views=12, width=128, height=96, f=110.0, dist=1.0)
    n, vox = 48, 0.5 / 48
    origin = c - 0.25
    F, W, amb = T.integrate(np.zeros((n, n, n)), np.zeros((n, n, n)), origin, vox, 0.04, 100.0, 0.5, cams, D, A)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    p = origin + (np.stack([i, j, k], -1) + 0.5) * vox
    r = np.linalg.norm(p - c, axis=-1)
    seen = W > 0
    assert seen.sum() > 1000
    outside = seen & (r > R + 1.5 * vox) & (r < R + 0.03)
    inside = seen & (r < R - 1.5 * vox) & (r > R - 0.03)
    assert (F[outside] > 0).mean() > 0.99 and (F[inside] < 0).mean() > 0.99
    assert not seen[r < R - 0.05].any()                  # deep inside: behind every surface by > trunc


def _one_voxel(centre, depth=1.0, trunc=0.25, vox=0.02):
    origin = np.asarray(centre, np.float64) - vox / 2
    return T.integrate(np.zeros((1, 1, 1)), np.zeros((1, 1, 1)), origin, vox, trunc, 100.0, 0.5, [CAM],
                       [np.full((32, 32), depth)], [np.ones((32, 32))])


def test_decisions_on_their_thresholds_are_flagged():
    """One voxel per case puts one integer decision of the fusion exactly on its threshold (the
    camera has f = 40, c = 16, so u = 40 x / z + 16): the oracle must flag it, since an FP32
    evaluation may take either side; an off-threshold control is not flagged and is updated in
    closed form (sdf = 1 - 1.2 = -0.2, f = -0.8, weight 1)."""
    for what, centre in [("pixel edge, u = 20", [0.1, 0.0125, 1.0]),
                         ("image border, u = 0", [-0.4, 0.0125, 1.0]),
                         ("sdf = -trunc", [0.015625, 0.015625, 1.25]),
                         ("camera plane, z = 0", [0.1, 0.0, 0.0])]:
        assert _one_voxel(centre)[2].all(), what
    F, W, amb = _one_voxel([0.015, 0.015, 1.2])
    assert not amb.any()
    assert W[0, 0, 0] == 1.0 and abs(F[0, 0, 0] + 0.8) < 1e-12
