"""Pixel-by-pixel comparison of a GPU render with the oracle's branches.

Tolerances (fixed by the method's statement of accuracy): max-abs 2e-3 per RGB channel and on
the coverage A = 1 - T, and 1e-4 relative on the depth of the pixel's surface.  Depth D is
unnormalised (sum of w_i z_i), so a coverage difference moves it by (A - A*) times the
surface depth D*/A*; that part is bounded by the coverage check and the remainder must satisfy
|D - D*| - |A - A*| D*/A* <= 1e-4 max(|D*|, 1e-6).  A pixel passes if it matches the oracle's
primary branch or one of its alternative branches (decisions within the FP32 error band taken
the other way); the oracle's extra tolerance for unexplored flips is added to every bound.
"""
import numpy as np

TOL_RGB = 2e-3
TOL_DREL = 1e-4
D_FLOOR = 1e-6


def _ok(g_rgb, g_d, g_a, rgb, d, a, tol_rgb, tol_d):
    e_rgb = np.abs(g_rgb - rgb).max(axis=-1)
    e_a = np.abs(g_a - a)
    surface = np.where(a > 1e-12, np.abs(d) / np.maximum(a, 1e-12), 0.0)
    e_d = np.abs(g_d - d)
    return (e_rgb <= TOL_RGB + tol_rgb) & (e_a <= TOL_RGB + tol_rgb) & \
        (e_d <= TOL_DREL * np.maximum(np.abs(d), D_FLOOR) + e_a * surface + tol_d)


def compare_view(g_rgb, g_depth, ref, g_alpha):
    """Returns (n_bad, report) for one view; g_* are [H,W,3] / [H,W] numpy arrays."""
    ok = _ok(g_rgb, g_depth, g_alpha, ref.rgb, ref.depth, ref.alpha, ref.tol_rgb, ref.tol_d)
    flat_ok = ok.reshape(-1)
    alt_used = 0
    bad_list = []
    for p in np.nonzero(~flat_ok)[0]:
        alts = ref.alternatives(int(p))
        y, x = divmod(int(p), ref.depth.shape[1])
        for a in alts:
            if _ok(g_rgb[y, x], g_depth[y, x], g_alpha[y, x], a[:3], a[3], a[4], ref.tol_rgb[y, x], ref.tol_d[y, x]):
                flat_ok[p] = True
                alt_used += 1
                break
        if not flat_ok[p] and len(bad_list) < 5:
            bad_list.append(dict(x=x, y=y, gpu=[*map(float, g_rgb[y, x]), float(g_depth[y, x]), float(g_alpha[y, x])],
                                 oracle=[*map(float, ref.rgb[y, x]), float(ref.depth[y, x]), float(ref.alpha[y, x])],
                                 n_alt=int(ref.n_alt[y, x])))
    bad = int((~flat_ok).sum())
    prim = ref.n_alt == 0
    surface = np.where(ref.alpha > 1e-12, np.abs(ref.depth) / np.maximum(ref.alpha, 1e-12), 0.0)
    d_excess = np.abs(g_depth - ref.depth) - np.abs(g_alpha - ref.alpha) * surface
    rep = dict(bad=bad, pixels=int(ok.size), ambiguous=ref.ambiguous_pixels, alt_used=alt_used,
               ambiguous_by_kind=ref.ambiguous_by_kind,
               max_rgb_err_unambiguous=float(np.abs(g_rgb - ref.rgb).max(axis=-1)[prim].max(initial=0.0)),
               max_alpha_err_unambiguous=float(np.abs(g_alpha - ref.alpha)[prim].max(initial=0.0)),
               max_depth_rel_err_unambiguous=float((np.maximum(d_excess, 0) /
                                                    np.maximum(np.abs(ref.depth), D_FLOOR))[prim].max(initial=0.0)),
               first_bad=bad_list)
    return bad, rep
