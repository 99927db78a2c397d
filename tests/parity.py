"""Pixel-by-pixel comparison of a GPU render with the oracle's branches.

Tolerances: max-abs 2e-3 per RGB channel (the method's stated accuracy), the same on the coverage
A = 1 - T, and 1e-4 relative on depth.

Depth D = sum_i w_i z_i is unnormalised, and A = sum_i w_i over the same weights.  A GPU whose
weights differ by dw_i therefore moves D by exactly (A - A*) D*/A* (the coverage change at the
pixel's mean depth D*/A*) plus sum_i dw_i (z_i - D*/A*) (the change of the depth distribution).
The 1e-4 relative bound applies to the second part.  The first part is admitted only as far as
the oracle's FP32 error model of the coverage explains it: the slack is min(|A - A*|, e_A) D*/A*,
with e_A = 2 T dT the FP32 error bound of A that the oracle carries along each branch
(dT = the relative error bound of the transmittance accumulated over the composited
Gaussians).  So a pixel passes when
    |C - C*| <= 2e-3,   |A - A*| <= 2e-3,
    |D - D*| <= 1e-4 max(|D*|, 1e-6) + min(|A - A*|, e_A) |D*| / A*
on the oracle's primary branch or one of its alternative branches (decisions within the FP32
error band taken the other way, the branch's own e_A); the oracle's extra tolerance for flips
beyond its branch budget is added to every bound.  Every report also gives the plain relative
depth error |D - D*| / max(|D*|, 1e-6) without the coverage term.
"""
import numpy as np

TOL_RGB = 2e-3
TOL_DREL = 1e-4
D_FLOOR = 1e-6


def _ok(g_rgb, g_d, g_a, rgb, d, a, ea, tol_rgb, tol_d):
    e_rgb = np.abs(g_rgb - rgb).max(axis=-1)
    e_a = np.abs(g_a - a)
    surface = np.where(a > 1e-12, np.abs(d) / np.maximum(a, 1e-12), 0.0)
    e_d = np.abs(g_d - d)
    return (e_rgb <= TOL_RGB + tol_rgb) & (e_a <= TOL_RGB + tol_rgb) & \
        (e_d <= TOL_DREL * np.maximum(np.abs(d), D_FLOOR) + np.minimum(e_a, ea) * surface + tol_d)


def compare_view(g_rgb, g_depth, ref, g_alpha):
    """Returns (n_bad, report) for one view; g_* are [H,W,3] / [H,W] numpy arrays."""
    ok = _ok(g_rgb, g_depth, g_alpha, ref.rgb, ref.depth, ref.alpha, ref.err_a, ref.tol_rgb, ref.tol_d)
    flat_ok = ok.reshape(-1)
    alt_used = 0
    bad_list = []
    for p in np.nonzero(~flat_ok)[0]:
        alts = ref.alternatives(int(p))
        y, x = divmod(int(p), ref.depth.shape[1])
        for a in alts:
            if _ok(g_rgb[y, x], g_depth[y, x], g_alpha[y, x], a[:3], a[3], a[4], a[5], ref.tol_rgb[y, x],
                   ref.tol_d[y, x]):
                flat_ok[p] = True
                alt_used += 1
                break
        if not flat_ok[p] and len(bad_list) < 5:
            bad_list.append(dict(x=x, y=y, gpu=[*map(float, g_rgb[y, x]), float(g_depth[y, x]), float(g_alpha[y, x])],
                                 oracle=[*map(float, ref.rgb[y, x]), float(ref.depth[y, x]), float(ref.alpha[y, x])],
                                 err_a=float(ref.err_a[y, x]), n_alt=int(ref.n_alt[y, x])))
    bad = int((~flat_ok).sum())
    prim = (ref.n_alt == 0) & (ref.tol_rgb == 0)
    d_rel = np.abs(g_depth - ref.depth) / np.maximum(np.abs(ref.depth), D_FLOOR)
    rep = dict(bad=bad, pixels=int(ok.size), ambiguous=ref.ambiguous_pixels, alt_used=alt_used,
               widened=ref.widened_pixels, ambiguous_by_kind=ref.ambiguous_by_kind,
               max_rgb_err_unambiguous=float(np.abs(g_rgb - ref.rgb).max(axis=-1)[prim].max(initial=0.0)),
               max_alpha_err_unambiguous=float(np.abs(g_alpha - ref.alpha)[prim].max(initial=0.0)),
               max_depth_rel_err_plain_unambiguous=float(d_rel[prim].max(initial=0.0)),
               frac_depth_plain_over_1e4_unambiguous=float((d_rel[prim] > TOL_DREL).mean()) if prim.any() else 0.0,
               max_err_a_bound=float(ref.err_a.max(initial=0.0)),
               first_bad=bad_list)
    return bad, rep
