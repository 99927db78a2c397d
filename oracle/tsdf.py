"""FP64 oracle of depth -> TSDF fusion.  Test infrastructure only: tests and the benchmark's CPU
baseline call it; the library never does.

Sec. III-B converts a Gaussian node back to a mesh by rendering multi-view depth maps and
fusing them into a truncated signed distance field (KinectFusion-style integration; the
decimation that follows is not part of this).  The definition taken here, per voxel centre
p = origin + (i + 1/2, j + 1/2, k + 1/2) * voxel (x fastest), per view in the given order:
  x_c = R p + t (cam_from_world); skip if z_c <= 0;
  (u, v) = (fx x_c / z_c + cx, fy y_c / z_c + cy); the pixel is (floor u, floor v) (the pixel
  whose area holds the projection; its centre is at +1/2); skip if outside the image;
  the measurement is the renderer's depth normalised by its coverage, d = D / A, valid only
  where A >= min_alpha; skip otherwise;
  sdf = d - z_c (along the optical axis); skip if sdf < -trunc (far behind the surface);
  f = min(1, sdf / trunc);
  F <- (W F + f) / (W + 1), W <- min(W + 1, max_weight).
Decisions an FP32 evaluation may take the other way are reported per voxel: a projection within
`band_px` of a pixel edge or of the image border, z_c within band of 0, or sdf within band of
-trunc (band relative to the magnitudes involved).
"""
from __future__ import annotations

import numpy as np


def integrate(tsdf, weight, origin, voxel: float, trunc: float, max_weight: float, min_alpha: float, cams,
              depth_views, alpha_views, band_px: float = 1e-3, band_rel: float = 1e-5):
    """Sec. III-B: fuses depth views into the field (definition in the module header).
    tsdf, weight: FP64 [nz, ny, nx] (updated copies are returned); cams: list of
    (fx, fy, cx, cy, W, H, cam_from_world [3,4]); depth_views / alpha_views: per view [H, W]
    (unnormalised D and coverage A).  Returns (tsdf, weight, ambiguous [nz, ny, nx] bool)."""
    F = np.array(tsdf, np.float64, copy=True)
    Wt = np.array(weight, np.float64, copy=True)
    nz, ny, nx = F.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    o = np.asarray(origin, np.float64)
    p = np.stack([o[0] + (i + 0.5) * voxel, o[1] + (j + 0.5) * voxel, o[2] + (k + 0.5) * voxel], axis=-1)
    amb = np.zeros(F.shape, bool)
    for (fx, fy, cx, cy, w_img, h_img, P), D, A in zip(cams, depth_views, alpha_views):
        P = np.asarray(P, np.float64)
        xc = p @ P[:, :3].T + P[:, 3]
        z = xc[..., 2]
        front = z > 0
        zs = np.where(front, z, 1.0)
        u = fx * xc[..., 0] / zs + cx
        v = fy * xc[..., 1] / zs + cy
        ui, vi = np.floor(u), np.floor(v)
        inside = front & (ui >= 0) & (ui < w_img) & (vi >= 0) & (vi < h_img)
        # ambiguity of the integer decisions
        zb = band_rel * (np.abs(xc).max(axis=-1) + 1.0)
        amb |= np.abs(z) <= zb
        near_edge = (np.abs(u - np.round(u)) <= band_px) | (np.abs(v - np.round(v)) <= band_px)
        amb |= front & near_edge & (u > -1) & (u < w_img + 1) & (v > -1) & (v < h_img + 1)
        uc = np.clip(ui, 0, w_img - 1).astype(np.int64)
        vc = np.clip(vi, 0, h_img - 1).astype(np.int64)
        Dp = np.asarray(D, np.float64)[vc, uc]
        Ap = np.asarray(A, np.float64)[vc, uc]
        valid = inside & (Ap >= min_alpha)
        d = np.where(valid, Dp / np.where(valid, Ap, 1.0), 0.0)
        sdf = d - z
        sb = band_rel * (np.abs(d) + np.abs(z) + trunc)
        amb |= valid & (np.abs(sdf + trunc) <= sb)
        upd = valid & (sdf >= -trunc)
        f = np.minimum(1.0, sdf / trunc)
        F = np.where(upd, (Wt * F + f) / (Wt + 1.0), F)
        Wt = np.where(upd, np.minimum(Wt + 1.0, max_weight), Wt)
    return F, Wt, amb
