"""Writes the golden fixtures of this folder: small, fully stated inputs together with the FP64
oracle's outputs for them, one JSON file per workload.

The script calls nothing but oracle/: its inputs are drawn here from seeded numpy generators
(and stored in the fixture, FP32-exact, next to the outputs), so no stored value comes from the
CUDA library.  The paper prints no worked example for any of these paths, so the fixtures are
regression anchors of the oracle, not independent pins (the pins are the closed forms,
invariants and brute-force cases of tests/test_oracle_*.py).  A change of the oracle's
arithmetic that moves a stored value regenerates the files in the same commit, which names
the passage that justifies it.

    python tests/golden/make_golden.py        # from the repository root
"""
from __future__ import annotations

import json
import os
import sys
from types import SimpleNamespace

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402

F32 = np.float32


def _f32(x) -> list:
    """FP32-exact nested list (every value is representable, so reading it back is lossless)."""
    return np.asarray(x, F32).astype(np.float64).tolist()


def _unit_quat(rng, n):
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _look_at_origin(yaw: float, dist: float) -> np.ndarray:
    """cam_from_world [3,4] of a camera on a circle of radius dist around the y axis, looking at
    the origin (OpenCV axes: x right, y down, z forward); its translation is (0, 0, dist)."""
    s, c = np.sin(yaw), np.cos(yaw)
    R = np.array([[c, 0.0, -s], [0.0, 1.0, 0.0], [s, 0.0, c]])
    return np.concatenate([R, np.array([[0.0], [0.0], [dist]])], axis=1)


# ----------------------------------------------------------------------------- scenes
def scene_from_inputs(inp: dict) -> SimpleNamespace:
    """The duck-typed scene the oracle reads, rebuilt from a fixture's stored inputs."""
    nodes = []
    for nd in inp["nodes"]:
        mean = np.asarray(nd["mean"], F32).reshape(-1, 3)
        n = len(mean)
        deg = int(nd["sh_degree"])
        nodes.append(SimpleNamespace(mean=mean, log_scale=np.asarray(nd["log_scale"], F32).reshape(n, 3),
                                     quat=np.asarray(nd["quat"], F32).reshape(n, 4),
                                     opacity_logit=np.asarray(nd["opacity_logit"], F32).reshape(n),
                                     sh=np.asarray(nd["sh"], F32).reshape(n, (deg + 1) ** 2, 3), sh_degree=deg, n=n))
    ids = np.asarray(inp["env_node_ids"], np.int32)
    E, K = ids.shape
    cpe = np.asarray(inp["cams_per_env"], np.int32)
    C = int(np.asarray(inp["cam_res"]).shape[1])
    return SimpleNamespace(nodes=nodes, env_node_ids=ids,
                           node_poses=np.asarray(inp["node_poses"], F32).reshape(E, K, 3, 4), cams_per_env=cpe,
                           cam_intr=np.asarray(inp["cam_intr"], F32).reshape(E, C, 4),
                           cam_res=np.asarray(inp["cam_res"], np.int32).reshape(E, C, 2),
                           cam_pose=np.asarray(inp["cam_pose"], F32).reshape(E, C, 3, 4),
                           views=[(e, c) for e in range(E) for c in range(int(cpe[e]))])


def _scene_inputs(seed: int = 11) -> dict:
    """Two nodes (a 6-Gaussian SH-degree-1 background, a 4-Gaussian SH-degree-0 object), two
    envs holding them in opposite slot orders at different object poses, and three cameras of
    three resolutions (8x6, 7x5, 6x4): a ragged batch of posed nodes."""
    rng = np.random.default_rng(seed)

    def node(n, deg, spread, ls_mu):
        return dict(mean=_f32(rng.uniform(-spread, spread, (n, 3))),
                    log_scale=_f32(rng.normal(ls_mu, 0.3, (n, 3))),
                    quat=_f32(rng.normal(size=(n, 4))),                     # unnormalised on purpose
                    opacity_logit=_f32(rng.normal(0.8, 1.0, n)),
                    sh=_f32(rng.normal(0.0, 0.4, (n, (deg + 1) ** 2, 3))), sh_degree=deg)

    bg, obj = node(6, 1, 0.6, -1.6), node(4, 0, 0.25, -1.9)
    poses = np.zeros((2, 2, 3, 4))
    poses[:, :, :, :3] = np.eye(3)
    for e, slot in ((0, 1), (1, 0)):                                        # the object's slot
        poses[e, slot, :, :3] = _rot(_unit_quat(rng, 1)[0])
        poses[e, slot, :, 3] = rng.uniform(-0.2, 0.2, 3)
    res = np.array([[[8, 6], [0, 0]], [[7, 5], [6, 4]]])
    intr = np.zeros((2, 2, 4))
    cpose = np.zeros((2, 2, 3, 4))
    for e, c, yaw in ((0, 0, 0.0), (1, 0, 0.5), (1, 1, -0.7)):
        w, h = res[e, c]
        intr[e, c] = (1.1 * w, 1.1 * w, w / 2, h / 2)
        cpose[e, c] = _look_at_origin(yaw, 3.0)
    return dict(nodes=[bg, obj], env_node_ids=[[0, 1], [1, 0]], node_poses=_f32(poses), cams_per_env=[1, 2],
                cam_intr=_f32(intr), cam_res=res.tolist(), cam_pose=_f32(cpose))


# ----------------------------------------------------------------------------- workloads
def render_fixture() -> dict:
    inp = _scene_inputs()
    sc = scene_from_inputs(inp)
    rng = np.random.default_rng(12)
    gr = [rng.normal(size=(int(sc.cam_res[e, c, 1]), int(sc.cam_res[e, c, 0]), 3)) for e, c in sc.views]
    gd = [rng.normal(size=g.shape[:2]) for g in gr]
    inp["grad_rgb"] = [g.tolist() for g in gr]
    inp["grad_depth"] = [g.tolist() for g in gd]
    return dict(cite="Sec. III-A (tile rasterisation, SH colour, front-to-back alpha compositing) and Sec. III-C "
                     "(depth composited from camera-space z); the adjoint is the analytic FP64 derivative of both",
                inputs=inp, expected=compute_render(inp))


def compute_render(inp: dict) -> dict:
    sc = scene_from_inputs(inp)
    views = []
    amb = 0
    for e, c in sc.views:
        r = O.render_view(sc, e, c)
        amb += r.ambiguous_pixels
        views.append(dict(rgb=r.rgb.tolist(), depth=r.depth.tolist(), alpha=r.alpha.tolist()))
    g = O.backward_scene(sc, [np.asarray(x) for x in inp["grad_rgb"]], [np.asarray(x) for x in inp["grad_depth"]])
    grads = {k: np.asarray(v).tolist() for k, v in g.items()}
    return dict(views=views, grads=grads, ambiguous_pixels=int(amb))


def lidar_fixture() -> dict:
    rng = np.random.default_rng(13)
    inp = _scene_inputs()
    poses = np.zeros((3, 3, 4))
    for s in range(3):
        q = np.concatenate([[1.0], rng.normal(0.0, 0.12, 3)]) if s else np.array([1.0, 0.0, 0.0, 0.0])
        poses[s, :, :3] = _rot(q / np.linalg.norm(q))                      # tilted forward views
        poses[s, :, 3] = (rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1), -1.5)
    phi = np.array([0.0, 0.08, 0.08, 0.08, 0.08, 0.2, 0.2, 0.2, 0.2, 0.35, 0.35, 0.35])
    psi = np.array([0.0, 0.0, 1.6, 3.1, 4.7, 0.8, 2.4, 3.9, 5.5, 0.3, 2.3, 4.4])
    dirs = np.stack([np.sin(phi) * np.cos(psi), np.sin(phi) * np.sin(psi), np.cos(phi)], axis=1)
    inp.update(sensor_env=[0, 1, 1], sensor_pose=_f32(poses), dirs=_f32(dirs), r_min=0.05, r_max=30.0)
    return dict(cite="Sec. III-C (LiDAR simulated by ray tracing the scene's Gaussians): per return the range sum "
                     "of weight x peak-response distance and the opacity 1 - T, hits composited nearest first",
                inputs=inp, expected=compute_lidar(inp))


def compute_lidar(inp: dict) -> dict:
    sc = scene_from_inputs(inp)
    r = O.lidar.trace(sc, np.asarray(inp["sensor_env"], np.int32), np.asarray(inp["sensor_pose"], F32).reshape(-1, 3, 4),
                      np.asarray(inp["dirs"], F32), O.lidar.LidarOptions(r_min=inp["r_min"], r_max=inp["r_max"]))
    return dict(d=r.d.tolist(), a=r.a.tolist(), n_comp=r.n_comp.tolist(), ambiguous=int(r.n_amb.sum()))


def augment_fixture() -> dict:
    rng = np.random.default_rng(14)
    rgb = rng.uniform(-0.1, 1.1, (4, 5, 3))
    rgb[0, 0] = 0.6                              # grey: zero chroma
    rgb[0, 1] = (1.0, 0.0, 0.0)                  # saturated red: hue at the wrap point
    rgb[1, 0] = (0.0, 0.0, 0.0)                  # black
    overlay = rng.integers(0, 256, (2, 3, 4, 3))
    params = [dict(hue_shift=0.04, sat_scale=1.2, val_scale=0.9, gamma=1.3, overlay_beta=0.3, overlay_frame=1,
                   overlay_x=2, overlay_y=1),
              dict(hue_shift=-0.03, sat_scale=0.8, val_scale=1.1, gamma=0.8, overlay_beta=0.0, overlay_frame=0,
                   overlay_x=0, overlay_y=0)]
    params = [{k: (float(F32(v)) if isinstance(v, float) else v) for k, v in p.items()} for p in params]
    inp = dict(rgb=_f32(rgb), overlay=overlay.tolist(), params=params)
    return dict(cite="Sec. IV (domain randomisation of rendered images: a moving-video overlay, HSV colour jitter "
                     "and gamma), applied in the order clamp, overlay blend, hexcone HSV jitter, gamma",
                inputs=inp, expected=compute_augment(inp))


def compute_augment(inp: dict) -> dict:
    rgb = np.asarray(inp["rgb"], F32)
    ov = np.asarray(inp["overlay"], np.uint8)
    return dict(out=[O.augment.augment_view(rgb, p, ov).tolist() for p in inp["params"]])


def mesh_fixture() -> dict:
    rng = np.random.default_rng(15)
    v = np.array([[0.0, 0.0, 0.0], [0.3, 0.0, 0.0], [0.0, 0.25, 0.0], [0.0, 0.0, 0.2],
                  [0.5, 0.5, 0.5], [0.6, 0.5, 0.5], [0.7, 0.5, 0.5]]) + rng.uniform(-1, 1, 3)
    f = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3],      # a closed tetrahedron, outward winding
                  [4, 5, 6],                                       # collinear: zero area
                  [4, 4, 5]])                                      # repeated vertex
    col = rng.uniform(0, 1, (len(v), 3))
    inp = dict(vertices=_f32(v), faces=f.tolist(), vertex_colors=_f32(col), flatten=0.02, opacity_logit=1.5,
               sh_degree=1)
    return dict(cite="Sec. III-B (mesh-to-Gaussian transfer: one flat Gaussian per facet at its barycentre, "
                     "aligned with its normal, tangent scale from the barycentre-to-vertex distances)",
                inputs=inp, expected=compute_mesh(inp))


def compute_mesh(inp: dict) -> dict:
    g = O.mesh.mesh_to_gaussians(np.asarray(inp["vertices"], F32), np.asarray(inp["faces"], np.int64),
                                 np.asarray(inp["vertex_colors"], F32), inp["flatten"], inp["opacity_logit"],
                                 inp["sh_degree"])
    return {k: np.asarray(g[k]).tolist() for k in ("mean", "log_scale", "quat", "opacity_logit", "sh")}


def tsdf_fixture() -> dict:
    rng = np.random.default_rng(16)
    nx, ny, nz = 5, 4, 3
    cams, D, A = [], [], []
    for yaw in (0.0, 0.6, -0.5, 2.9):
        w, h = 7, 6
        cams.append((6.0, 6.0, 3.5, 3.0, w, h, _f32(_look_at_origin(yaw, 1.0))))
        depth = 1.0 + rng.uniform(-0.2, 0.2, (h, w))
        alpha = rng.choice([0.0, 0.3, 0.8, 1.0], (h, w))
        D.append(_f32(depth * alpha))
        A.append(_f32(alpha))
    inp = dict(shape=[nz, ny, nx], tsdf0=_f32(rng.uniform(-1, 1, (nz, ny, nx))),
               weight0=_f32(rng.integers(0, 3, (nz, ny, nx))), origin=_f32([-0.2437, -0.1913, -0.1571]), voxel=0.0937,
               trunc=0.15, max_weight=3.0, min_alpha=0.5,
               cams=[dict(fx=c[0], fy=c[1], cx=c[2], cy=c[3], width=c[4], height=c[5], cam_from_world=c[6])
                     for c in cams], depth=D, alpha=A)
    inp["voxel"], inp["trunc"] = float(F32(0.0937)), float(F32(0.15))
    return dict(cite="Sec. III-B (rendered multi-view depth fused into a truncated signed distance field before "
                     "meshing): projective sdf along the optical axis, truncation, weighted running average",
                inputs=inp, expected=compute_tsdf(inp))


def compute_tsdf(inp: dict) -> dict:
    cams = [(c["fx"], c["fy"], c["cx"], c["cy"], c["width"], c["height"], np.asarray(c["cam_from_world"], F32))
            for c in inp["cams"]]
    F, W, amb = O.tsdf.integrate(np.asarray(inp["tsdf0"], F32), np.asarray(inp["weight0"], F32), inp["origin"],
                                 inp["voxel"], inp["trunc"], inp["max_weight"], inp["min_alpha"], cams,
                                 [np.asarray(d, F32) for d in inp["depth"]], [np.asarray(a, F32) for a in inp["alpha"]])
    return dict(tsdf=F.tolist(), weight=W.tolist(), ambiguous=int(amb.sum()))


FIXTURES = {"render_two_envs": (render_fixture, compute_render), "lidar_three_sensors": (lidar_fixture, compute_lidar),
            "augment_two_params": (augment_fixture, compute_augment), "mesh_tetra_degenerate": (mesh_fixture, compute_mesh),
            "tsdf_four_views": (tsdf_fixture, compute_tsdf)}


def path(name: str) -> str:
    return os.path.join(HERE, name + ".json")


def main() -> None:
    O.build()
    for name, (make, _) in FIXTURES.items():
        fx = make()
        ex = fx["expected"]
        for k in ("ambiguous_pixels", "ambiguous"):
            assert ex.get(k, 0) == 0, f"{name}: inputs meet {ex[k]} ambiguous decisions; pick another seed"
        fx = dict(name=name, generator="tests/golden/make_golden.py (calls only oracle/)", **fx)
        with open(path(name), "w") as fh:
            json.dump(fx, fh, separators=(",", ":"))
            fh.write("\n")
        print(name, os.path.getsize(path(name)), "bytes")


if __name__ == "__main__":
    main()
