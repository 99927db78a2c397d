"""Golden fixtures (tests/golden/*.json): small, fully stated inputs of every workload (the
batched render and its adjoint, LiDAR, the image randomisation, the mesh transfer, TSDF fusion)
with the FP64 oracle's outputs, written by tests/golden/make_golden.py, which calls only the
oracle.  They anchor the oracle against unnoticed drift: recomputing each fixture must give
the stored values to 1e-9 relative (the files are shared by machines whose libm and FMA
contraction differ in the last bits).  Every fixture cites the passage it follows, its inputs
are FP32-exact, and none of them meets an ambiguous FP32 decision, so a device-side comparison
against the stored values needs no branch enumeration.  No GPU is needed.
"""
import json

import numpy as np
import pytest

from tests.golden import make_golden as G


def _load(name):
    with open(G.path(name)) as fh:
        return json.load(fh)


def _close(got, want, what):
    if isinstance(want, dict):
        assert set(got) == set(want), what
        for k in want:
            _close(got[k], want[k], f"{what}.{k}")
    elif isinstance(want, list) and want and isinstance(want[0], dict):
        assert len(got) == len(want), what
        for i, (g, w) in enumerate(zip(got, want)):
            _close(g, w, f"{what}[{i}]")
    else:
        g, w = np.asarray(got, np.float64), np.asarray(want, np.float64)
        assert g.shape == w.shape, (what, g.shape, w.shape)
        scale = max(1.0, float(np.abs(w).max(initial=0.0)))
        np.testing.assert_allclose(g, w, rtol=1e-9, atol=1e-12 * scale, err_msg=what)


@pytest.mark.parametrize("name", sorted(G.FIXTURES))
def test_oracle_reproduces_fixture(name):
    fx = _load(name)
    _, compute = G.FIXTURES[name]
    _close(compute(fx["inputs"]), fx["expected"], name)


@pytest.mark.parametrize("name", sorted(G.FIXTURES))
def test_fixture_is_cited_exact_and_unambiguous(name):
    fx = _load(name)
    assert fx["name"] == name and fx["cite"].startswith("Sec. ") and "oracle" in fx["generator"]
    ex = fx["expected"]
    assert ex.get("ambiguous_pixels", 0) == 0 and ex.get("ambiguous", 0) == 0
    inp = fx["inputs"]
    floats = []
    for nd in inp.get("nodes", []):
        floats += [nd[k] for k in ("mean", "log_scale", "quat", "opacity_logit", "sh")]
    floats += [inp[k] for k in ("node_poses", "cam_intr", "cam_pose", "sensor_pose", "dirs", "rgb", "vertices",
                                "vertex_colors", "tsdf0", "weight0", "origin", "depth", "alpha") if k in inp]
    for x in floats:
        a = np.asarray(x, np.float64)
        assert np.array_equal(a.astype(np.float32).astype(np.float64), a)


def test_fixtures_exercise_their_paths():
    """Guards against fixtures that pass vacuously: covered pixels and non-zero gradients in
    every view, a return on most LiDAR beams of every sensor, both overlay states, a degenerate
    facet with the identity frame, and TSDF voxels both updated and capped."""
    r = _load("render_two_envs")["expected"]
    for v in r["views"]:
        assert (np.asarray(v["alpha"]) > 0.05).mean() > 0.5
    for k in ("mean", "log_scale", "quat", "opacity_logit", "sh", "pose"):
        assert np.abs(np.asarray(r["grads"][k])).max() > 1e-3, k
    lid = _load("lidar_three_sensors")["expected"]
    assert ((np.asarray(lid["a"]) > 0.05).mean(axis=1) > 0.8).all()
    aug = _load("augment_two_params")["inputs"]["params"]
    assert {p["overlay_beta"] > 0 for p in aug} == {True, False}
    mesh = _load("mesh_tetra_degenerate")["expected"]
    np.testing.assert_array_equal(np.asarray(mesh["quat"])[4:], [[1, 0, 0, 0]] * 2)
    t = _load("tsdf_four_views")
    w0, w1 = np.asarray(t["inputs"]["weight0"]), np.asarray(t["expected"]["weight"])
    assert (w1 > w0).any() and (w1 == t["inputs"]["max_weight"]).any() and (w1 == w0).any()
