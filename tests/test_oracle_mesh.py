"""Pins of the mesh -> Gaussian oracle (oracle/mesh.py) against facts that do not come from it:
an equilateral facet's closed form, the covariance's eigen-decomposition against the facet's
normal from an SVD of its vertices, the quaternion against scipy's rotations, rigid-motion
equivariance, winding, the colour round trip, degenerate facets, and the FP64 camera oracle
rendering a converted square opaque inside its outline.  No GPU is needed.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from oracle import mesh as M
from paper_2507_21981_gb300 import scenes as S


def test_equilateral_facet_closed_form():
    a = 0.3
    v = np.array([[0, 0, 0], [a, 0, 0], [a / 2, a * math.sqrt(3) / 2, 0]], np.float64) + [1.0, 2.0, 3.0]
    g = M.mesh_to_gaussians(v, np.array([[0, 1, 2]]), flatten=0.05)
    np.testing.assert_allclose(g["mean"][0], v.mean(axis=0), atol=1e-15)
    s = a / math.sqrt(3)                         # circumradius = barycentre-to-vertex distance
    np.testing.assert_allclose(g["log_scale"][0], np.log([s, s, 0.05 * s]), atol=1e-14)
    np.testing.assert_allclose(M.covariance(g["log_scale"], g["quat"])[0], np.diag([s * s, s * s, (0.05 * s) ** 2]),
                               atol=1e-15)
    np.testing.assert_allclose(g["rot"][0][:, 2], [0, 0, 1], atol=1e-15)    # counter-clockwise: +z


def test_covariance_eigensystem_against_svd_normal():
    v, f = S.mesh_icosphere(2, 0.2)
    rng = np.random.default_rng(0)
    v = v + rng.normal(0, 0.01, v.shape).astype(np.float32)
    g = M.mesh_to_gaussians(v, f, flatten=0.02)
    cov = M.covariance(g["log_scale"], g["quat"])
    for i in rng.choice(len(f), 40, replace=False):
        p = v[f[i]].astype(np.float64)
        c = p - p.mean(axis=0)
        n_svd = np.linalg.svd(c)[2][2]           # direction of zero spread of the facet
        w, vec = np.linalg.eigh(cov[i])
        st = np.mean(np.linalg.norm(c, axis=1))
        np.testing.assert_allclose(w, [(0.02 * st) ** 2, st * st, st * st], rtol=1e-10)
        assert abs(abs(vec[:, 0] @ n_svd) - 1) < 1e-10


def test_quaternion_matches_scipy():
    v, f = S.mesh_icosphere(1, 1.0)
    g = M.mesh_to_gaussians(v, f)
    q = g["quat"]
    Rs = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], axis=1)).as_matrix()
    np.testing.assert_allclose(Rs, g["rot"], atol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-14)


def test_rigid_equivariance_and_winding():
    v, f, _ = S.mesh_heightfield(1, 12, 9)
    v = v.astype(np.float64)
    g = M.mesh_to_gaussians(v, f)
    P = S.random_pose(np.random.default_rng(2), 1.0)
    g2 = M.mesh_to_gaussians(v @ P[:, :3].T + P[:, 3], f)
    np.testing.assert_allclose(g2["mean"], g["mean"] @ P[:, :3].T + P[:, 3], atol=1e-12)
    c1, c2 = M.covariance(g["log_scale"], g["quat"]), M.covariance(g2["log_scale"], g2["quat"])
    np.testing.assert_allclose(c2, P[:, :3] @ c1 @ P[:, :3].T, atol=1e-14)
    gr = M.mesh_to_gaussians(v, f[:, ::-1])       # reversed winding: normal flips, covariance stays
    np.testing.assert_allclose(gr["rot"][:, :, 2], -g["rot"][:, :, 2], atol=1e-12)
    np.testing.assert_allclose(M.covariance(gr["log_scale"], gr["quat"]), c1, atol=1e-14)


def test_colour_round_trip_and_degenerate_facet():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [2, 2, 2]], np.float64)
    col = np.array([[0.1, 0.2, 0.3], [0.5, 0.5, 0.5], [0.9, 0.8, 0.1], [0, 0, 0]])
    f = np.array([[0, 1, 2], [3, 3, 3], [0, 1, 1]])
    g = M.mesh_to_gaussians(v, f, vertex_colors=col, sh_degree=2)
    np.testing.assert_allclose(0.5 + M.Y00 * g["sh"][0, 0], col[:3].mean(axis=0), atol=1e-15)
    assert np.all(g["sh"][:, 1:] == 0) and g["sh"].shape == (3, 9, 3)
    assert np.allclose(g["rot"][1], np.eye(3)) and np.allclose(g["rot"][2], np.eye(3))
    assert np.all(np.isfinite(g["log_scale"]))
    assert g["log_scale"][1, 0] == pytest.approx(math.log(1e-12))


def test_converted_square_renders_opaque_inside_its_outline():
    """A 1 m square (16 x 16 grid) converted with opaque facets and viewed head-on: the FP64
    camera oracle sees coverage ~1 well inside the square and 0 well outside it."""
    v, f, col = S.mesh_heightfield(3, 17, 17, size=1.0, amp=0.0)
    g = M.mesh_to_gaussians(v, f, vertex_colors=col, flatten=0.01, opacity_logit=6.0)
    f32 = np.float32
    node = S.GaussianNode(g["mean"].astype(f32), g["log_scale"].astype(f32), g["quat"].astype(f32),
                          g["opacity_logit"].astype(f32), g["sh"].astype(f32), 0, "mesh")
    cam = S.look_at([0.5, 0.5, 1.5], [0.5, 0.5, 0.0], up=(0.0, 1.0, 0.0))
    sc = S.scene_from_lists("sq", [node], [[0]], [[np.eye(3, 4)]], [[(64.0, 64.0, 32.0, 32.0, 64, 64, cam)]])
    r = O.render_view(sc, 0, 0, O.OracleOptions(nthreads=2))
    # the square spans about 64 * 1 / 1.5 = 43 px around the centre
    inner = r.alpha[22:42, 22:42]
    assert inner.min() > 0.99
    assert r.alpha[:4].max() < 1e-6 and r.alpha[:, :4].max() < 1e-6
    # coplanar facets composite in id order: the colour is a convex mix of facet colours
    inside = r.rgb[22:42, 22:42].reshape(-1, 3)
    assert (inside >= col.min(axis=0) - 1e-3).all() and (inside <= col.max(axis=0) + 1e-3).all()
