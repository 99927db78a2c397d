"""The seeded input generators (scenes.py) produce what the tests and the benchmark assume: the
LiDAR beam pattern in 4 x 8 tiles of unit directions, rigid sensor poses near the workspace,
overlay clips and randomisation parameters in their ranges, closed outward-wound icospheres,
upward heightfields, and sphere depth maps whose back-projected pixels lie on the sphere.  The
benchmark's reference arm prints one JSON line with the contract's keys.  No GPU is needed.
"""
import json
import os
import subprocess
import sys

import numpy as np

from paper_2507_21981_gb300 import scenes as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_lidar_pattern_tiles_and_units():
    d = S.lidar_pattern(32, 1024)
    assert d.shape == (32 * 1024, 3) and d.dtype == np.float32
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    plain = S.lidar_pattern(32, 1024, tile=None)
    # the tiled order is a permutation of the same float32 beams: recover (channel, azimuth)
    where = {plain[k].tobytes(): divmod(k, 1024) for k in range(len(plain))}
    ca = np.array([where[x.tobytes()] for x in d])
    assert len({tuple(x) for x in ca}) == len(d)
    for p in range(0, len(d), 32):                      # every 32 consecutive beams: one 4 x 8 tile
        c, a = ca[p:p + 32, 0], ca[p:p + 32, 1]
        assert c.max() - c.min() == 3 and a.max() - a.min() == 7


def test_lidar_sensors_rigid_near_workspace():
    env, pose = S.lidar_sensors(3, 16)
    assert env.tolist() == list(range(16))
    R = pose[:, :, :3].astype(np.float64)
    np.testing.assert_allclose(R @ R.transpose(0, 2, 1), np.broadcast_to(np.eye(3), R.shape), atol=1e-5)
    r = np.linalg.norm(pose[:, :2, 3] - S.WORKSPACE_CENTRE[:2], axis=1)
    assert (r >= 1.0 - 1e-5).all() and (r <= 2.0 + 1e-5).all()
    assert (pose[:, 2, 3] >= 0.8).all() and (pose[:, 2, 3] <= 1.6).all()


def test_overlay_and_parameter_ranges():
    ov = S.overlay_frames(2, n_frames=3, width=96, height=64)
    assert ov.shape == (3, 64, 96, 3) and ov.dtype == np.uint8
    assert ov.std() > 20 and len(np.unique(ov)) > 100            # textured, not flat
    assert not np.array_equal(ov[0], ov[1])                     # frames differ (moving content)
    p = S.augment_params(5, 500, 3, 96, 64)
    assert (np.abs(p["hue_shift"]) <= 0.05).all()
    assert ((p["sat_scale"] >= 0.7) & (p["sat_scale"] <= 1.3)).all()
    assert ((p["gamma"] >= 0.7) & (p["gamma"] <= 1.5)).all()
    on = p["overlay_beta"] > 0
    assert 0.35 < on.mean() < 0.65 and ((p["overlay_beta"][on] >= 0.1) & (p["overlay_beta"][on] <= 0.4)).all()
    assert (p["overlay_frame"] < 3).all() and (p["overlay_x"] < 96).all() and (p["overlay_y"] < 64).all()


def test_icosphere_closed_and_outward():
    v, f = S.mesh_icosphere(2, 0.3)
    assert len(f) == 20 * 4 ** 2
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 0.3, rtol=1e-6)
    p0, p1, p2 = (v[f[:, k]].astype(np.float64) for k in range(3))
    vol = np.einsum("ij,ij->i", p0, np.cross(p1, p2)).sum() / 6.0       # signed volume: outward winding > 0
    assert abs(vol - 4 / 3 * np.pi * 0.3 ** 3) < 0.05 * 4 / 3 * np.pi * 0.3 ** 3
    edges = np.sort(np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]]), axis=1)
    _, counts = np.unique(edges, axis=0, return_counts=True)
    assert (counts == 2).all()                                         # closed 2-manifold


def test_heightfield_upward_and_coloured():
    v, f, col = S.mesh_heightfield(1, 20, 15, size=2.0, amp=0.05)
    assert len(f) == 2 * 19 * 14 and v.shape == (300, 3) and col.shape == (300, 3)
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    assert (n[:, 2] > 0).all()
    assert (col >= 0).all() and (col <= 1).all()


def test_sphere_depth_back_projects_onto_the_sphere():
    c, R = np.array([0.2, -0.1, 0.4]), 0.25
    cams, D, A = S.sphere_depth_views(c, R, n_views=3, width=40, height=30, f=35.0, dist=1.0, seed=4)
    for (fx, fy, cx, cy, w, h, P), d, a in zip(cams, D, A):
        ys, xs = np.nonzero(a > 0)
        assert len(ys) > 50 and (a[a > 0] == 1).all()
        z = d[ys, xs].astype(np.float64)
        xc = np.stack([(xs + 0.5 - cx) / fx * z, (ys + 0.5 - cy) / fy * z, z], axis=1)
        P = np.asarray(P, np.float64)
        pw = (xc - P[:, 3]) @ P[:, :3]                                    # world = R^T (x_c - t)
        np.testing.assert_allclose(np.linalg.norm(pw - c, axis=1), R, atol=1e-4)


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "cpu_baseline",
              "e2e", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
