"""The renderer's parity criterion (tests/parity.py: 2e-3 on RGB and coverage, 1e-4 relative on
depth, any of the oracle's branches accepted) is tight enough to catch plausible mistakes.

Each mistake is expressed through the oracle's inputs or options, rendered by the oracle itself
in FP64 and scored against the correct render with the criterion the GPU tests apply.  The
mistakes follow the readings of the paper they would break:
- no screen-space low-pass (R2);
- pixels sampled at integer coordinates (R7);
- quaternions read as (x, y, z, w) (R12);
- log-scales taken as log-variances;
- node poses ignored (Sec. III-B: object Gaussians move with their node);
- SH without the Condon-Shortley phase (R10);
- depth normalised by coverage (R5);
- alpha not clamped at 0.99 (R4).
No GPU is needed.
"""
import copy

import numpy as np
import pytest

import oracle as O
from paper_2507_21981_gb300 import scenes as S
from tests.parity import compare_view

BASE = O.OracleOptions(nthreads=4)


def _opts(**kw):
    d = dict(BASE.__dict__)
    d.update(kw)
    return O.OracleOptions(**d)


def _scene(logit_shift=0.0):
    """A 64x64 view of a 3k-Gaussian background and a posed 1k-Gaussian object, SH degree 3."""
    sc = S.config1(seed=3, n_bg=3000, n_obj=1000, res=64, f=55.0)
    rng = np.random.default_rng(4)
    for nd in sc.nodes:
        sh = rng.normal(0.0, 0.25, (nd.n, 16, 3)).astype(np.float32)
        sh[:, 0] = nd.sh[:, 0]
        nd.sh, nd.sh_degree = sh, 3
        nd.opacity_logit = (nd.opacity_logit + np.float32(logit_shift)).astype(np.float32)
    return sc


def _shift_centres(s):
    s.cam_intr = s.cam_intr.copy()
    s.cam_intr[..., 2:] += 0.5


def _quat_xyzw(s):
    for nd in s.nodes:
        nd.quat = np.ascontiguousarray(nd.quat[:, [1, 2, 3, 0]])


def _log_variance(s):
    for nd in s.nodes:
        nd.log_scale = (nd.log_scale * np.float32(0.5)).astype(np.float32)


def _no_pose(s):
    s.node_poses = np.zeros_like(s.node_poses)
    s.node_poses[..., :3] = np.eye(3)


def _no_cs_phase(s):
    for nd in s.nodes:
        for l in range(1, 4):
            for m in range(-l, l + 1):
                if abs(m) % 2:
                    nd.sh[:, l * l + l + m] *= -1


MISTAKES = {
    "no low-pass": (None, dict(lowpass=0.0)),
    "integer pixel centres": (_shift_centres, {}),
    "quaternion as xyzw": (_quat_xyzw, {}),
    "log-scale as log-variance": (_log_variance, {}),
    "node pose ignored": (_no_pose, {}),
    "SH without Condon-Shortley phase": (_no_cs_phase, {}),
}


@pytest.fixture(scope="module")
def reference():
    sc = _scene()
    return sc, O.render_view(sc, 0, 0, BASE)


def _bad(ref, g_rgb, g_depth, g_alpha):
    bad, _ = compare_view(g_rgb, g_depth, ref, g_alpha)
    return bad


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_mistake_fails_most_covered_pixels(reference, name):
    sc, ref = reference
    mutate, kw = MISTAKES[name]
    s2 = copy.deepcopy(sc)
    if mutate:
        mutate(s2)
    g = O.render_view(s2, 0, 0, _opts(**kw) if kw else BASE)
    covered = int((ref.alpha > 0.05).sum())
    assert covered > 0.9 * ref.alpha.size
    assert _bad(ref, g.rgb, g.depth, g.alpha) > 0.5 * covered, name     # measured: 97-100 %


def test_depth_normalised_by_coverage_fails(reference):
    _, ref = reference
    d = np.where(ref.alpha > 0, ref.depth / np.maximum(ref.alpha, 1e-12), 0.0)
    assert _bad(ref, ref.rgb, d, ref.alpha) > 0.5 * (ref.alpha > 0.05).sum()


def test_missing_alpha_clamp_fails_near_opaque_centres():
    """Only pixels within about 0.14 sigma of an opaque Gaussian's centre reach the clamp, so the
    mistake shows on a few dozen pixels of an opaque scene (measured 30); the GPU tests fail on
    any bad pixel."""
    sc = _scene(logit_shift=6.0)
    ref = O.render_view(sc, 0, 0, BASE)
    g = O.render_view(sc, 0, 0, _opts(alpha_max=1.0))
    assert _bad(ref, g.rgb, g.depth, g.alpha) >= 10
