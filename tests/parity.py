"""Pixel-by-pixel comparison of a GPU render with the oracle's branches.

Tolerances (fixed by the method's statement of accuracy): max-abs 2e-3 per RGB channel and
1e-4 relative depth, |D - D*| <= 1e-4 * max(|D*|, 1e-6).  A pixel passes if it matches the
oracle's primary branch or one of its alternative branches (decisions within the FP32
ambiguity band taken the other way); the oracle's extra tolerance for unexplored flips is
added to both bounds.
"""
import numpy as np

TOL_RGB = 2e-3
TOL_DREL = 1e-4
D_FLOOR = 1e-6


def _ok(g_rgb, g_d, rgb, d, tol_rgb, tol_d):
    e_rgb = np.abs(g_rgb - rgb).max(axis=-1)
    e_d = np.abs(g_d - d)
    return (e_rgb <= TOL_RGB + tol_rgb) & (e_d <= TOL_DREL * np.maximum(np.abs(d), D_FLOOR) + tol_d)


def compare_view(g_rgb, g_depth, ref, g_alpha=None):
    """Returns (n_bad, report) for one view; g_* are [H,W,3] / [H,W] numpy arrays."""
    ok = _ok(g_rgb, g_depth, ref.rgb, ref.depth, ref.tol_rgb, ref.tol_d)
    if g_alpha is not None:
        ok &= np.abs(g_alpha - ref.alpha) <= TOL_RGB + ref.tol_rgb
    flat_ok = ok.reshape(-1)
    alt_used = 0
    for p in np.nonzero(~flat_ok)[0]:
        alts = ref.alternatives(int(p))
        if len(alts) == 0:
            continue
        y, x = divmod(int(p), ref.depth.shape[1])
        for a in alts:
            good = _ok(g_rgb[y, x], g_depth[y, x], a[:3], a[3], ref.tol_rgb[y, x], ref.tol_d[y, x])
            if g_alpha is not None:
                good = good and abs(g_alpha[y, x] - a[4]) <= TOL_RGB + ref.tol_rgb[y, x]
            if good:
                flat_ok[p] = True
                alt_used += 1
                break
    bad = int((~flat_ok).sum())
    prim = ref.n_alt == 0
    rep = dict(bad=bad, pixels=int(ok.size), ambiguous=ref.ambiguous_pixels, alt_used=alt_used,
               max_rgb_err_unambiguous=float(np.abs(g_rgb - ref.rgb).max(axis=-1)[prim].max(initial=0.0)),
               max_depth_rel_err_unambiguous=float((np.abs(g_depth - ref.depth) /
                                                    np.maximum(np.abs(ref.depth), D_FLOOR))[prim].max(initial=0.0)))
    return bad, rep
