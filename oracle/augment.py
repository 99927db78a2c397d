"""FP64 oracle of the image randomisation applied to rendered frames.  Test infrastructure
only: tests, the smoke check and the benchmark's CPU baseline call it; the library never does.

Sec. IV ("Sim2Real" data generation) trains policies on rendered frames that are randomised in
three ways: crops of Internet videos linearly blended into the frame, jitter in HSV space, and
a random gamma correction.  The paper fixes neither the order nor the parameterisation; the
reading taken here (one parameter set per view, drawn by the caller) is

    c0 = clamp(rgb, 0, 1)                                      rendered colour, clamped
    c1 = (1 - beta) c0 + beta o                                overlay blend
         o = overlay[f, (oy + y) mod OH, (ox + x) mod OW] / 255   (crop with wrap-around)
    (H, S, V) = hsv(c1)                                        hexcone model (Smith, 1978)
    H' = frac(H + hue_shift), S' = min(1, S sat_scale), V' = min(1, V val_scale)
    c2 = rgb(H', S', V')
    out = c2 ** gamma                                          (0 ** gamma = 0)

The overlay is blended first because it stands for something in front of the camera; the HSV
jitter and the gamma curve stand for the camera's colour response and act on everything it
sees.  Depth is not randomised.  Every step is written out in the textbook form of the hexcone
model, H in turns (one turn = 360 degrees).
"""
from __future__ import annotations

import numpy as np

# field order of one view's parameters
FIELDS = ("hue_shift", "sat_scale", "val_scale", "gamma", "overlay_beta", "overlay_frame", "overlay_x",
          "overlay_y")


def rgb_to_hsv(c: np.ndarray) -> np.ndarray:
    """Sec. IV (HSV colour jitter), RGB -> HSV.  Hexcone model: V = max, C = max - min, S = C / V (0
    for V = 0), H from the sector of the largest channel (red checked first, then green), in turns
    in [0, 1); H = 0 for C = 0. c: [..., 3] -> [..., 3] (H, S, V)."""
    c = np.asarray(c, dtype=np.float64)
    r, g, b = c[..., 0], c[..., 1], c[..., 2]
    v = np.maximum(np.maximum(r, g), b)
    m = np.minimum(np.minimum(r, g), b)
    chroma = v - m
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(v > 0, chroma / np.where(v > 0, v, 1.0), 0.0)
        safe = np.where(chroma > 0, chroma, 1.0)
        h_r = ((g - b) / safe) % 6.0
        h_g = (b - r) / safe + 2.0
        h_b = (r - g) / safe + 4.0
    h = np.where(v == r, h_r, np.where(v == g, h_g, h_b))
    h = np.where(chroma > 0, h / 6.0, 0.0)
    return np.stack([h, s, v], axis=-1)


def hsv_to_rgb(hsv: np.ndarray) -> np.ndarray:
    """Sec. IV (HSV colour jitter), HSV -> RGB.  Inverse hexcone map: sector i = floor(6H) mod 6,
    fraction f = 6H - floor(6H), p = V(1 - S), q = V(1 - S f), t = V(1 - S(1 - f)), and per sector
    (V,t,p) (q,V,p) (p,V,t) (p,q,V) (t,p,V) (V,p,q).  hsv: [..., 3] -> [..., 3]."""
    hsv = np.asarray(hsv, dtype=np.float64)
    h, s, v = hsv[..., 0], hsv[..., 1], hsv[..., 2]
    h6 = h * 6.0
    fl = np.floor(h6)
    f = h6 - fl
    i = fl.astype(np.int64) % 6
    p = v * (1.0 - s)
    q = v * (1.0 - s * f)
    t = v * (1.0 - s * (1.0 - f))
    table = [(v, t, p), (q, v, p), (p, v, t), (p, q, v), (t, p, v), (v, p, q)]
    out = np.zeros(h.shape + (3,), dtype=np.float64)
    for k, (rr, gg, bb) in enumerate(table):
        sel = i == k
        out[..., 0] = np.where(sel, rr, out[..., 0])
        out[..., 1] = np.where(sel, gg, out[..., 1])
        out[..., 2] = np.where(sel, bb, out[..., 2])
    return out


def overlay_crop(overlay: np.ndarray, frame: int, ox: int, oy: int, w: int, h: int) -> np.ndarray:
    """Sec. IV (blend with crops of video frames).  The w x h crop of overlay frame `frame` whose pixel
    (x, y) is frame pixel ((oy + y) mod OH, (ox + x) mod OW), as FP64 in [0, 1].  overlay: uint8 [F,
    OH, OW, 3]."""
    n_f, oh, ow, _ = overlay.shape
    assert 0 <= frame < n_f
    rows = (oy + np.arange(h)) % oh
    cols = (ox + np.arange(w)) % ow
    return overlay[frame][np.ix_(rows, cols)].astype(np.float64) / 255.0


def augment_view(rgb: np.ndarray, prm, overlay: np.ndarray | None, return_stages: bool = False):
    """Sec. IV: randomises one rendered view.  rgb: [H, W, 3] (any float type; taken as FP64);
    prm: mapping or record with the FIELDS above; overlay: uint8 [F, OH, OW, 3] (may be None
    when overlay_beta == 0).  Returns out [H, W, 3] FP64 (and, with return_stages, a dict of
    the intermediate images c0, c1, c2)."""
    rgb = np.asarray(rgb, dtype=np.float64)
    h_img, w_img = rgb.shape[:2]
    beta = float(prm["overlay_beta"])
    c0 = np.clip(rgb, 0.0, 1.0)
    if beta != 0.0:
        o = overlay_crop(overlay, int(prm["overlay_frame"]), int(prm["overlay_x"]), int(prm["overlay_y"]),
                         w_img, h_img)
        c1 = (1.0 - beta) * c0 + beta * o
    else:
        c1 = c0
    hsv = rgb_to_hsv(c1)
    hue = hsv[..., 0] + float(prm["hue_shift"])
    hue = hue - np.floor(hue)
    sat = np.minimum(1.0, hsv[..., 1] * float(prm["sat_scale"]))
    val = np.minimum(1.0, hsv[..., 2] * float(prm["val_scale"]))
    c2 = hsv_to_rgb(np.stack([hue, sat, val], axis=-1))
    out = c2 ** float(prm["gamma"])
    if return_stages:
        return out, dict(c0=c0, c1=c1, c2=c2)
    return out


def gamma_spread(c2: np.ndarray, gamma: float, delta: float) -> np.ndarray:
    """Sec. IV (random gamma), tolerance helper.  Largest change of c ** gamma when c (in [0, 1]) moves
    by at most delta: the error that an absolute error delta before the gamma curve can leave after
    it.  Used to state tolerances; c ** gamma is monotone, so the extremes sit at c +- delta."""
    c2 = np.asarray(c2, dtype=np.float64)
    hi = np.minimum(c2 + delta, 1.0) ** gamma
    lo = np.maximum(c2 - delta, 0.0) ** gamma
    mid = c2 ** gamma
    return np.maximum(hi - mid, mid - lo)
