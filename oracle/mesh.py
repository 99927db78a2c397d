"""FP64 oracle of the mesh -> Gaussian transfer.  Test infrastructure only: tests and the
benchmark's CPU baseline call it; the library never does.

Sec. III-B (Mesh-Gaussian Transfer): every facet of a textured mesh becomes one Gaussian
centred on the facet's barycentre, flattened to a planar primitive whose local frame is aligned
with the facet's normal, with both tangent-axis scales set to the facet's mean
barycentre-to-vertex distance.  Readings where the paper is silent:
  * normal n = (v1 - v0) x (v2 - v0) / |...| (the facet's winding); the tangent frame is
    (t1, t2, n) with t1 = (v1 - v0)/|v1 - v0| and t2 = n x t1 (the in-plane rotation does not
    change the covariance, the two tangent scales being equal);
  * the normal-axis scale is flatten x the tangent scale (a 3D renderer needs a non-zero width;
    flatten is an input);
  * opacity and colour are the optimisation's starting point, not geometry: the opacity logit
    is an input, the degree-0 SH coefficient is (c - 1/2) / Y_00 with c the mean of the facet's
    vertex colours (or 1/2 without colours, i.e. zero), higher-degree coefficients zero;
  * a facet of zero area keeps the identity frame; tangent scales below 1e-12 are raised to it.
Outputs follow the renderer's node layout: mean [F,3], log_scale [F,3] (natural logs of the
standard deviations, order t1, t2, n), quat [F,4] (w, x, y, z), opacity_logit [F],
sh [F, (deg+1)^2, 3].
"""
from __future__ import annotations

import math

import numpy as np

Y00 = 0.5 / math.sqrt(math.pi)     # real SH basis, degree 0


def facet_frames(v: np.ndarray, f: np.ndarray):
    """Sec. III-B (mesh-Gaussian transfer).  Per facet: barycentre b, tangent scale s_t, rotation R
    (columns t1, t2, n) and a flag for zero-area facets.  v [V,3], f [F,3] int."""
    v = np.asarray(v, np.float64)
    p0, p1, p2 = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    b = (p0 + p1 + p2) / 3.0
    s_t = (np.linalg.norm(p0 - b, axis=1) + np.linalg.norm(p1 - b, axis=1) + np.linalg.norm(p2 - b, axis=1)) / 3.0
    s_t = np.maximum(s_t, 1e-12)
    e1, e2 = p1 - p0, p2 - p0
    cr = np.cross(e1, e2)
    area2 = np.linalg.norm(cr, axis=1)
    l1 = np.linalg.norm(e1, axis=1)
    degenerate = (area2 == 0) | (l1 == 0)
    R = np.tile(np.eye(3), (len(f), 1, 1))
    ok = ~degenerate
    n = cr[ok] / area2[ok, None]
    t1 = e1[ok] / l1[ok, None]
    t2 = np.cross(n, t1)
    R[ok] = np.stack([t1, t2, n], axis=2)
    return b, s_t, R, degenerate


def quat_from_rot(R: np.ndarray) -> np.ndarray:
    """Sec. III-B: the facet frame as the node layout's quaternion.  (w, x, y, z) of rotation matrices
    [F,3,3] (Shepperd's method: the largest of the four squared components decides), sign chosen
    with w >= 0."""
    F = len(R)
    q = np.zeros((F, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    cand = np.stack([tr, R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], axis=1)
    k = np.argmax(cand, axis=1)
    for i in range(F):
        m = R[i]
        if k[i] == 0:
            s = math.sqrt(1.0 + tr[i]) * 2
            q[i] = [0.25 * s, (m[2, 1] - m[1, 2]) / s, (m[0, 2] - m[2, 0]) / s, (m[1, 0] - m[0, 1]) / s]
        elif k[i] == 1:
            s = math.sqrt(1.0 + m[0, 0] - m[1, 1] - m[2, 2]) * 2
            q[i] = [(m[2, 1] - m[1, 2]) / s, 0.25 * s, (m[0, 1] + m[1, 0]) / s, (m[0, 2] + m[2, 0]) / s]
        elif k[i] == 2:
            s = math.sqrt(1.0 + m[1, 1] - m[0, 0] - m[2, 2]) * 2
            q[i] = [(m[0, 2] - m[2, 0]) / s, (m[0, 1] + m[1, 0]) / s, 0.25 * s, (m[1, 2] + m[2, 1]) / s]
        else:
            s = math.sqrt(1.0 + m[2, 2] - m[0, 0] - m[1, 1]) * 2
            q[i] = [(m[1, 0] - m[0, 1]) / s, (m[0, 2] + m[2, 0]) / s, (m[1, 2] + m[2, 1]) / s, 0.25 * s]
    q *= np.where(q[:, :1] < 0, -1.0, 1.0)
    return q


def mesh_to_gaussians(v, f, vertex_colors=None, flatten: float = 0.01, opacity_logit: float = 2.0,
                      sh_degree: int = 0) -> dict:
    """Sec. III-B: the transfer of every facet (see the module header).  Returns a dict of FP64 arrays."""
    f = np.asarray(f, np.int64)
    b, s_t, R, _ = facet_frames(v, f)
    F = len(f)
    log_scale = np.stack([np.log(s_t), np.log(s_t), np.log(flatten * s_t)], axis=1)
    nc = (sh_degree + 1) ** 2
    sh = np.zeros((F, nc, 3))
    if vertex_colors is not None:
        c = np.asarray(vertex_colors, np.float64)
        mc = (c[f[:, 0]] + c[f[:, 1]] + c[f[:, 2]]) / 3.0
        sh[:, 0, :] = (mc - 0.5) / Y00
    return dict(mean=b, log_scale=log_scale, quat=quat_from_rot(R), opacity_logit=np.full(F, float(opacity_logit)),
                sh=sh, rot=R)


def covariance(log_scale: np.ndarray, quat: np.ndarray) -> np.ndarray:
    """Sec. III-A (3DGS covariance from scale and rotation): Sigma = R diag(exp(2 log_scale)) R^T for
    (w, x, y, z) quaternions (normalised here)."""
    q = np.asarray(quat, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                  np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                  np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], axis=1)
    s2 = np.exp(2 * np.asarray(log_scale, np.float64))
    return np.einsum("fij,fj,fkj->fik", R, s2, R)
