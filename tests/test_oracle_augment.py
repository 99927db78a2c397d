"""Pins of the image-randomisation oracle (oracle/augment.py) against facts that do not come
from the oracle itself: Python's colorsys (an independent implementation of the hexcone
model), closed forms of special parameter values (a hue shift of a third of a turn permutes
the channels, zero saturation gives the grey of the largest channel, value scaling is a plain
scaling, gamma on greys is a power), the overlay crop read back pixel by pixel, and the order
of the three steps.  No GPU is needed.
"""
import colorsys

import numpy as np
import pytest

from oracle import augment as A
from paper_2507_21981_gb300 import scenes as S

IDENT = dict(hue_shift=0.0, sat_scale=1.0, val_scale=1.0, gamma=1.0, overlay_beta=0.0, overlay_frame=0,
             overlay_x=0, overlay_y=0)


def prm(**kw):
    d = dict(IDENT)
    d.update(kw)
    return d


def _colours(n=4000, seed=0):
    """Random colours plus the edge cases of the hexcone model: black, white, greys, primaries,
    secondaries, and ties between the largest channels."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, 1, size=(n, 3))
    edge = [[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1],
            [1, 0, 1], [0.7, 0.7, 0.2], [0.2, 0.7, 0.7], [0.7, 0.2, 0.7], [0.3, 0.1, 0.3], [1e-9, 0, 0],
            [0.25, 0.5, 0.5], [0.9, 0.9, 0.9 - 1e-12]]
    return np.concatenate([c, np.array(edge, dtype=np.float64)], axis=0)


def test_rgb_to_hsv_matches_colorsys():
    c = _colours()
    got = A.rgb_to_hsv(c)
    ref = np.array([colorsys.rgb_to_hsv(*row) for row in c])
    assert np.allclose(got, ref, atol=1e-12, rtol=0)


def test_hsv_to_rgb_matches_colorsys():
    rng = np.random.default_rng(1)
    hsv = rng.uniform(0, 1, size=(4000, 3))
    hsv[:50, 0] = np.arange(50) / 6.0 % 1.0          # sector boundaries
    hsv[50:60, 1] = 0.0
    hsv[60:70, 2] = 0.0
    got = A.hsv_to_rgb(hsv)
    ref = np.array([colorsys.hsv_to_rgb(*row) for row in hsv])
    assert np.allclose(got, ref, atol=1e-12, rtol=0)


def test_round_trip_is_identity():
    c = _colours()
    assert np.allclose(A.hsv_to_rgb(A.rgb_to_hsv(c)), c, atol=1e-12, rtol=0)


def _img(seed=2, h=9, w=13):
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.2, 1.3, size=(h, w, 3))      # out-of-range values exercise the clamp


def test_identity_parameters_only_clamp():
    x = _img()
    assert np.allclose(A.augment_view(x, prm(), None), np.clip(x, 0, 1), atol=1e-12, rtol=0)


@pytest.mark.parametrize("shift,perm", [(1 / 3, (2, 0, 1)), (2 / 3, (1, 2, 0)), (-1 / 3, (1, 2, 0)),
                                        (1.0, (0, 1, 2)), (-2.0, (0, 1, 2)), (4 / 3, (2, 0, 1))])
def test_hue_third_turns_permute_channels(shift, perm):
    """A hue rotation by 120 degrees maps red to green, green to blue and blue to red in the
    hexcone model: (r, g, b) -> (b, r, g); whole turns change nothing."""
    x = np.clip(_img(3), 0, 1)
    got = A.augment_view(x, prm(hue_shift=shift), None)
    assert np.allclose(got, x[..., list(perm)], atol=1e-12, rtol=0)


def test_zero_saturation_gives_grey_of_the_largest_channel():
    x = np.clip(_img(4), 0, 1)
    got = A.augment_view(x, prm(sat_scale=0.0), None)
    v = x.max(axis=-1, keepdims=True)
    assert np.allclose(got, np.broadcast_to(v, x.shape), atol=1e-12, rtol=0)


def test_value_scale_scales_colour():
    x = np.clip(_img(5), 0, 1) * 0.6
    got = A.augment_view(x, prm(val_scale=1.5), None)
    assert np.allclose(got, 1.5 * x, atol=1e-12, rtol=0)
    # above 1 the value saturates: the largest channel becomes exactly 1, hue and saturation stay
    y = np.array([[[0.8, 0.4, 0.2]]])
    assert np.allclose(A.augment_view(y, prm(val_scale=2.0), None), [[[1.0, 0.5, 0.25]]], atol=1e-12)


def test_saturation_scale_closed_form():
    """S -> S k keeps V and H: for c = (V, m, m) (pure red hue) the result is (V, V - k(V - m), same)."""
    y = np.array([[[0.8, 0.5, 0.5]]])
    k = 1.5
    assert np.allclose(A.augment_view(y, prm(sat_scale=k), None), [[[0.8, 0.8 - k * 0.3, 0.8 - k * 0.3]]],
                       atol=1e-12)
    # saturation clamps at 1: the smallest channel reaches 0
    assert np.allclose(A.augment_view(y, prm(sat_scale=10.0), None), [[[0.8, 0.0, 0.0]]], atol=1e-12)


def test_gamma_on_greys_is_a_power():
    g = np.linspace(0, 1, 11)
    x = np.stack([g, g, g], axis=-1)[None]
    for gam in (0.5, 0.8, 1.7):
        got = A.augment_view(x, prm(gamma=gam), None)
        assert np.allclose(got[0, :, 0], g ** gam, atol=1e-12)
        assert got[0, 0, 0] == 0.0


def _overlay():
    rng = np.random.default_rng(6)
    return rng.integers(0, 256, size=(3, 5, 7, 3), dtype=np.uint8)


def test_full_overlay_weight_shows_the_wrapped_crop():
    ov = _overlay()
    x = _img(7, h=6, w=9)                 # larger than the 5x7 frame: the crop wraps in both axes
    got = A.augment_view(x, prm(overlay_beta=1.0, overlay_frame=2, overlay_x=4, overlay_y=3), ov)
    for y in range(6):
        for xx in range(9):
            want = ov[2, (3 + y) % 5, (4 + xx) % 7] / 255.0
            assert np.allclose(got[y, xx], want, atol=1e-12)


def test_overlay_blend_is_linear():
    ov = _overlay()
    x = np.clip(_img(8, h=4, w=4), 0, 1)
    b = 0.25
    got = A.augment_view(x, prm(overlay_beta=b, overlay_frame=1, overlay_x=1, overlay_y=2), ov)
    o = ov[1][np.ix_([2, 3, 4, 0], [1, 2, 3, 4])] / 255.0    # rows (2 + y) mod 5, columns (1 + x) mod 7
    assert np.allclose(got, 0.75 * x + 0.25 * o, atol=1e-12)


def test_order_blend_then_hsv_then_gamma():
    """The overlay is blended before the colour jitter and the gamma curve act: with weight 1 the
    output is the jittered overlay; with a hue shift of a third of a turn and gamma 2 the
    channels of the blend are permuted, then squared."""
    ov = _overlay()
    x = np.clip(_img(9, h=5, w=7), 0, 1)
    o = ov[0] / 255.0
    got = A.augment_view(x, prm(overlay_beta=1.0, gamma=2.0), ov)
    assert np.allclose(got, o ** 2, atol=1e-12)
    got = A.augment_view(x, prm(overlay_beta=0.5, hue_shift=1 / 3, gamma=2.0), ov)
    blend = 0.5 * x + 0.5 * o
    assert np.allclose(got, blend[..., [2, 0, 1]] ** 2, atol=1e-12)


def test_outputs_stay_in_unit_range_for_drawn_parameters():
    ov = S.overlay_frames(3, n_frames=2, width=64, height=48)
    p = S.augment_params(3, 16, 2, 64, 48, p_overlay=0.7)
    x = _img(10, h=40, w=50)
    for k in range(16):
        out = A.augment_view(x, p[k], ov)
        assert out.min() >= 0.0 and out.max() <= 1.0 + 1e-15


def test_gamma_spread_bounds_the_power_curve():
    rng = np.random.default_rng(11)
    c = rng.uniform(0, 1, 2000)
    c[:5] = [0.0, 1e-9, 1e-4, 1.0, 0.5]
    for gam in (0.6, 1.0, 1.4):
        d = 1e-6
        s = A.gamma_spread(c, gam, d)
        for e in (-d, -d / 2, d / 2, d):
            moved = np.clip(c + e, 0, 1) ** gam
            assert np.all(np.abs(moved - c ** gam) <= s + 1e-15)
