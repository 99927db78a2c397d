"""Mesh -> Gaussian transfer on the GPU (dgs_mesh_to_gaussians) against the FP64 oracle.

Per facet: the mean within 4u of the coordinates' magnitude (u = 2^-24), the log-scales within
2e-6 (the kernel works from the edges, so the scale's error is relative to the facet's size), unit quaternions with w >= 0, the covariance R diag(s^2) R^T (the unique part: the
in-plane rotation is free) within s^2 (2 dtheta + 16u) with dtheta = 16u |e1||e2| / |e1 x e2|
the FP32 error of the normal's direction, the opacity logit exactly, the degree-0 SH coefficient
within 1e-5 and the higher ones exactly zero.  Cases: a noisy icosphere, a coloured heightfield
with SH degree 3, exactly degenerate facets, an index out of range, and 10k facets sampled from
a 1M-facet mesh.
"""
import numpy as np
import pytest

from oracle import mesh as M
from paper_2507_21981_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _gpu(v, f, col=None, **kw):
    from paper_2507_21981_gb300.render import Renderer
    r = Renderer()
    out = r.mesh_to_gaussians(torch.as_tensor(v).cuda(), torch.as_tensor(f).cuda(),
                              None if col is None else torch.as_tensor(col).cuda(), **kw)
    res = {k: t.cpu().numpy() for k, t in out.items()}
    r.close()
    return res


def _check(v, f, g, ref):
    v = np.asarray(v, np.float64)
    p0, p1, p2 = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    mag = np.abs(np.stack([p0, p1, p2])).max(axis=(0, 2))
    assert (np.abs(g["mean"] - ref["mean"]).max(axis=1) <= 4 * U * mag + 1e-30).all()
    assert np.abs(g["log_scale"] - ref["log_scale"]).max() <= 2e-6
    q = g["quat"].astype(np.float64)
    assert np.abs(np.linalg.norm(q, axis=1) - 1).max() < 2e-6 and (q[:, 0] >= 0).all()
    e1, e2 = p1 - p0, p2 - p0
    area2 = np.linalg.norm(np.cross(e1, e2), axis=1)
    cond = np.where(area2 > 0, np.linalg.norm(e1, axis=1) * np.linalg.norm(e2, axis=1) / np.maximum(area2, 1e-300), 1)
    s2 = np.exp(2 * ref["log_scale"][:, 0])
    tol = s2 * (2 * 16 * U * cond + 16 * U) + 1e-30
    err = np.abs(M.covariance(g["log_scale"], g["quat"]) - M.covariance(ref["log_scale"], ref["quat"])).max(axis=(1, 2))
    assert (err <= tol).all(), (float((err / tol).max()), int(np.argmax(err / tol)))
    assert np.array_equal(g["opacity_logit"], ref["opacity_logit"].astype(np.float32))
    assert np.abs(g["sh"][:, 0] - ref["sh"][:, 0]).max() <= 1e-5
    assert (g["sh"][:, 1:] == 0).all()


def test_noisy_icosphere():
    v, f = S.mesh_icosphere(3, 0.08)
    v = (v + np.random.default_rng(1).normal(0, 0.002, v.shape)).astype(np.float32)
    g = _gpu(v, f, flatten=0.02, opacity_logit=1.5)
    _check(v, f, g, M.mesh_to_gaussians(v, f, flatten=0.02, opacity_logit=1.5))


def test_coloured_heightfield_sh3():
    v, f, col = S.mesh_heightfield(2, 40, 31, size=2.0, amp=0.1)
    v = v + np.array([3.0, -1.0, 0.5], np.float32)          # away from the origin
    g = _gpu(v, f, col, sh_degree=3)
    _check(v, f, g, M.mesh_to_gaussians(v, f, vertex_colors=col, sh_degree=3))
    assert g["sh"].shape == (len(f), 16, 3)


def test_degenerate_facets_and_bad_index():
    v = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0], [0.5, 0.5, 1.0]], np.float32)
    f = np.array([[0, 1, 3], [0, 1, 2], [1, 1, 1], [0, 0, 3], [3, 4, 1]], np.int32)   # collinear, point, repeated
    g = _gpu(v, f)
    ref = M.mesh_to_gaussians(v, f)
    _check(v, f, g, ref)
    assert np.allclose(g["quat"][1:4], [1, 0, 0, 0])
    from paper_2507_21981_gb300 import dgs as D
    with pytest.raises(D.DgsError):
        _gpu(v, np.array([[0, 1, 5]], np.int32))
    with pytest.raises(D.DgsError):
        _gpu(v, np.array([[0, -1, 2]], np.int32))


def test_million_facet_mesh_sampled():
    v, f, col = S.mesh_heightfield(5, 708, 708, size=4.0, amp=0.2)
    g = _gpu(v, f, col, sh_degree=3)
    assert len(f) == 2 * 707 * 707
    assert np.isfinite(g["mean"]).all() and np.isfinite(g["log_scale"]).all() and np.isfinite(g["quat"]).all()
    idx = np.random.default_rng(3).choice(len(f), 10_000, replace=False)
    sub = {k: a[idx] for k, a in g.items()}
    _check(v, f[idx], sub, M.mesh_to_gaussians(v, f[idx], vertex_colors=col, sh_degree=3))
