"""Seeded synthetic scenes for the batched Gaussian-splatting renderer.

This module only *draws inputs*: Gaussian attributes of the scene nodes, the per-env
rigid node poses that a physics engine would supply, and the cameras. It contains none
of the renderer's arithmetic (no projection, colour evaluation, binning or compositing),
so both the CUDA path and the CPU oracle can be fed from it without sharing any of the
method's code.

Scene model (Sec. III-B "Asset Formatting" and Sec. III-C "Sensor"): every environment
holds a background node (3DGS only) plus interactive nodes (objects, robots) whose
Gaussians move rigidly with the pose of their node.  Poses are world_from_node 3x4
matrices; cameras are pinhole with OpenCV axes (x right, y down, z forward) and a
cam_from_world 3x4 extrinsic.

The paper's own scenes (laser-scanned rooms, scanned or generated objects, Sec. IV) are
not available; these generators stand in for them with the same structure: an indoor room
of a few hundred square metres of surface, a one-metre tabletop workspace holding small
objects, two to three cameras per environment (third-person, ego, side), 640x480 images.

Randomness: numpy's PCG64 seeded through SeedSequence(seed, spawn_key=(stream,)); every
draw is float64 and is rounded to float32 at the end, so a scene is a pure function of
(config, seed, size parameters).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

SH_COEFFS = {0: 1, 1: 4, 2: 9, 3: 16}
# Y_0^0 of the real spherical-harmonic basis: 1 / (2 sqrt(pi)).  Only used to store a
# requested degree-0 colour c as the coefficient (c - 0.5) / Y00.
_Y00 = 0.5 / math.sqrt(math.pi)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed, spawn_key=(stream,))))


@dataclass
class GaussianNode:
    """Structure-of-arrays Gaussians of one scene node, in the node's own frame."""
    mean: np.ndarray           # [N,3] float32
    log_scale: np.ndarray      # [N,3] float32, natural log of the std-devs along the local axes
    quat: np.ndarray           # [N,4] float32, (w,x,y,z), not necessarily unit
    opacity_logit: np.ndarray  # [N]   float32
    sh: np.ndarray             # [N,(deg+1)^2,3] float32, coefficient-major per Gaussian
    sh_degree: int
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def subset(self, idx) -> "GaussianNode":
        return GaussianNode(self.mean[idx].copy(), self.log_scale[idx].copy(), self.quat[idx].copy(),
                            self.opacity_logit[idx].copy(), self.sh[idx].copy(), self.sh_degree,
                            self.name)


@dataclass
class Scene:
    """A batch of environments x cameras over a set of shared nodes.

    env_node_ids[e, j] is the node drawn in slot j of env e (-1 = empty slot); a node id may
    appear at most once per env.  node_poses[e, j] is that node's world_from_node pose.
    Views are enumerated env-major: view v <-> (e, c) for c < cams_per_env[e].
    """
    name: str
    nodes: list
    env_node_ids: np.ndarray   # [E,K] int32
    node_poses: np.ndarray     # [E,K,3,4] float32
    cams_per_env: np.ndarray   # [E] int32
    cam_intr: np.ndarray       # [E,C,4] float32 (fx, fy, cx, cy)
    cam_res: np.ndarray        # [E,C,2] int32 (width, height)
    cam_pose: np.ndarray       # [E,C,3,4] float32 cam_from_world
    meta: dict = field(default_factory=dict)

    @property
    def n_envs(self) -> int:
        return int(self.env_node_ids.shape[0])

    @property
    def views(self):
        return [(e, c) for e in range(self.n_envs) for c in range(int(self.cams_per_env[e]))]

    @property
    def n_views(self) -> int:
        return int(self.cams_per_env.sum())

    def view_res(self, v: int):
        e, c = self.views[v]
        return int(self.cam_res[e, c, 0]), int(self.cam_res[e, c, 1])

    @property
    def n_pixels(self) -> int:
        return int(sum(self.cam_res[e, c, 0] * self.cam_res[e, c, 1] for e, c in self.views))

    @property
    def n_gaussians(self) -> int:
        return int(sum(nd.n for nd in self.nodes))

    def instances(self) -> int:
        """Sum over views of the Gaussians present in that view's env."""
        tot = 0
        for e, c in self.views:
            tot += sum(self.nodes[k].n for k in self.env_node_ids[e] if k >= 0)
        return int(tot)


# ----------------------------------------------------------------------------- rotations
def _uniform_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random unit quaternions, (w,x,y,z), by Shoemake's subgroup algorithm."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = b * np.sin(2 * np.pi * u3)
    w = b * np.cos(2 * np.pi * u3)
    return np.stack([w, x, y, z], axis=1)


def _qmul(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Hamilton product of (w,x,y,z) quaternions (broadcasting)."""
    pw, px, py, pz = np.moveaxis(p, -1, 0)
    qw, qx, qy, qz = np.moveaxis(q, -1, 0)
    return np.stack([pw * qw - px * qx - py * qy - pz * qz,
                     pw * qx + px * qw + py * qz - pz * qy,
                     pw * qy - px * qz + py * qw + pz * qx,
                     pw * qz + px * qy - py * qx + pz * qw], axis=-1)


def _rotmat_from_unit_quat(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of a unit quaternion; used only to build pose and camera inputs."""
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _rot_axis(axis: np.ndarray, angle: float) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    h = 0.5 * angle
    return _rotmat_from_unit_quat(np.array([math.cos(h), *(math.sin(h) * axis)]))


def _orthonormalise(R: np.ndarray) -> np.ndarray:
    u, _, vt = np.linalg.svd(R)
    Q = u @ vt
    if np.linalg.det(Q) < 0:
        u[:, -1] *= -1
        Q = u @ vt
    return Q


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """cam_from_world [R|t] (3x4) of a camera at `eye` looking at `target` (OpenCV axes)."""
    eye, target, up = (np.asarray(a, dtype=np.float64) for a in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    if abs(float(np.dot(f, up))) > 0.999:
        up = np.array([0.0, 1.0, 0.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)                      # image "down"
    R = np.stack([r, d, f])                 # rows: camera x, y, z axes in world coordinates
    return np.concatenate([R, (-R @ eye)[:, None]], axis=1)


def _jitter_camera(rng: np.random.Generator, P: np.ndarray, pos_m: float, rot_deg: float) -> np.ndarray:
    """Perturb a cam_from_world pose: centre by U[-pos,pos]^3, orientation by a small rotation."""
    R, t = P[:, :3], P[:, 3]
    centre = -R.T @ t + rng.uniform(-pos_m, pos_m, 3)
    ang = np.deg2rad(rng.uniform(-rot_deg, rot_deg, 3))
    dR = _rot_axis([1, 0, 0], ang[0]) @ _rot_axis([0, 1, 0], ang[1]) @ _rot_axis([0, 0, 1], ang[2])
    R2 = _orthonormalise(dR @ R)
    return np.concatenate([R2, (-R2 @ centre)[:, None]], axis=1)


# ----------------------------------------------------------------------------- nodes
def uniform_cube_node(rng: np.random.Generator, n: int, half: float, log_scale_mu: float,
                      log_scale_sd: float, opacity_mu: float, opacity_sd: float,
                      sh_degree: int, sh_sd: float | None = None, name: str = "") -> GaussianNode:
    """Means uniform in [-half, half]^3, iid normal log-scales, uniform rotations.

    Colour: for sh_degree 0 with sh_sd None, a colour c ~ U[0,1]^3 stored as (c-0.5)/Y00;
    otherwise every coefficient ~ N(0, sh_sd).
    """
    mean = rng.uniform(-half, half, (n, 3))
    log_scale = rng.normal(log_scale_mu, log_scale_sd, (n, 3))
    quat = _uniform_quats(rng, n)
    opacity_logit = rng.normal(opacity_mu, opacity_sd, n)
    ncoef = SH_COEFFS[sh_degree]
    if sh_sd is None:
        assert sh_degree == 0
        colour = rng.random((n, 3))
        sh = ((colour - 0.5) / _Y00)[:, None, :]
    else:
        sh = rng.normal(0.0, sh_sd, (n, ncoef, 3))
    f = np.float32
    return GaussianNode(mean.astype(f), log_scale.astype(f), quat.astype(f), opacity_logit.astype(f),
                        np.ascontiguousarray(sh.astype(f)), sh_degree, name)


def _room_surfaces(rng: np.random.Generator, size=(10.0, 10.0, 3.0), n_boxes=20):
    """Axis-aligned rectangles: floor, ceiling, four walls and the five visible faces of boxes.

    Each surface is (normal_axis, plane_coordinate, (lo_u, hi_u), (lo_v, hi_v)) where u, v
    are the two remaining axes in increasing order.
    """
    sx, sy, sz = size
    hx, hy = sx / 2, sy / 2
    surf = [(2, 0.0, (-hx, hx), (-hy, hy)), (2, sz, (-hx, hx), (-hy, hy)),
            (0, -hx, (-hy, hy), (0.0, sz)), (0, hx, (-hy, hy), (0.0, sz)),
            (1, -hy, (-hx, hx), (0.0, sz)), (1, hy, (-hx, hx), (0.0, sz))]
    for _ in range(n_boxes):
        cx, cy = rng.uniform(-hx + 0.7, hx - 0.7), rng.uniform(-hy + 0.7, hy - 0.7)
        ex, ey = rng.uniform(0.15, 0.6), rng.uniform(0.15, 0.6)
        h = rng.uniform(0.3, 1.5)
        x0, x1, y0, y1 = cx - ex, cx + ex, cy - ey, cy + ey
        surf += [(2, h, (x0, x1), (y0, y1)),
                 (0, x0, (y0, y1), (0.0, h)), (0, x1, (y0, y1), (0.0, h)),
                 (1, y0, (x0, x1), (0.0, h)), (1, y1, (x0, x1), (0.0, h))]
    return surf


# local z -> world axis, as unit quaternions (w,x,y,z)
_S = math.sqrt(0.5)
_ALIGN_Z_TO = {0: np.array([_S, 0.0, _S, 0.0]),    # rotate +90 deg about y: z -> x
               1: np.array([_S, -_S, 0.0, 0.0]),   # rotate -90 deg about x: z -> y
               2: np.array([1.0, 0.0, 0.0, 0.0])}


def room_node(rng: np.random.Generator, n: int, sh_degree: int = 3, size=(10.0, 10.0, 3.0),
              n_boxes: int = 20, normal_noise: float = 0.01, log_scale_mu: float = -4.0,
              log_scale_sd: float = 0.5, flatten: float = 0.1, opacity_mu: float = 1.0,
              opacity_sd: float = 1.5, sh_sd: float = 0.2, name: str = "room") -> GaussianNode:
    """Background node: Gaussians on noisy planes and boxes inside a room.

    Points are uniform on the surfaces (allocated by area) plus N(0, normal_noise) along the
    normal.  Each Gaussian's local z axis is the surface normal (random in-plane rotation)
    and its scale along that axis is multiplied by `flatten`.
    """
    surf = _room_surfaces(rng, size, n_boxes)
    areas = np.array([(u[1] - u[0]) * (v[1] - v[0]) for _, _, u, v in surf])
    counts = rng.multinomial(n, areas / areas.sum())
    means, quats = [], []
    for (axis, c, (u0, u1), (v0, v1)), m in zip(surf, counts):
        if m == 0:
            continue
        others = [a for a in range(3) if a != axis]
        p = np.empty((m, 3))
        p[:, others[0]] = rng.uniform(u0, u1, m)
        p[:, others[1]] = rng.uniform(v0, v1, m)
        p[:, axis] = c + rng.normal(0.0, normal_noise, m)
        means.append(p)
        psi = rng.uniform(0, 2 * np.pi, m)
        qz = np.stack([np.cos(psi / 2), np.zeros(m), np.zeros(m), np.sin(psi / 2)], axis=1)
        quats.append(_qmul(_ALIGN_Z_TO[axis][None, :], qz))
    mean = np.concatenate(means)
    quat = np.concatenate(quats)
    perm = rng.permutation(n)              # interleave surfaces in memory order
    mean, quat = mean[perm], quat[perm]
    log_scale = rng.normal(log_scale_mu, log_scale_sd, (n, 3))
    log_scale[:, 2] += math.log(flatten)
    opacity_logit = rng.normal(opacity_mu, opacity_sd, n)
    sh = rng.normal(0.0, sh_sd, (n, SH_COEFFS[sh_degree], 3))
    f = np.float32
    return GaussianNode(mean.astype(f), log_scale.astype(f), quat.astype(f), opacity_logit.astype(f),
                        np.ascontiguousarray(sh.astype(f)), sh_degree, name)


def object_node(rng: np.random.Generator, n: int, sh_degree: int = 3, name: str = "object") -> GaussianNode:
    """An interactive object: points in a 0.1 m box, log-scale N(-5.5, 0.5)."""
    return uniform_cube_node(rng, n, 0.05, -5.5, 0.5, 1.0, 1.5, sh_degree, 0.2, name)


# ----------------------------------------------------------------------------- poses, cameras
WORKSPACE_CENTRE = np.array([0.0, 0.0, 1.3])   # 1 m cube standing on a table top at z = 0.8 m


def workspace_pose(rng: np.random.Generator) -> np.ndarray:
    """world_from_node for an object in the workspace: yaw U[-pi,pi] then a tilt of N(0,5 deg)."""
    t = WORKSPACE_CENTRE + rng.uniform(-0.5, 0.5, 3)
    yaw = rng.uniform(-np.pi, np.pi)
    ax = rng.normal(size=2)
    tilt = np.deg2rad(rng.normal(0.0, 5.0))
    R = _rot_axis([ax[0], ax[1], 0.0], tilt) @ _rot_axis([0, 0, 1], yaw)
    return np.concatenate([R, t[:, None]], axis=1)


def random_pose(rng: np.random.Generator, t_half: float) -> np.ndarray:
    """Uniform rotation (Shoemake) and t ~ U[-t_half, t_half]^3."""
    R = _rotmat_from_unit_quat(_uniform_quats(rng, 1)[0])
    return np.concatenate([R, rng.uniform(-t_half, t_half, 3)[:, None]], axis=1)


def _third_person(rng):
    el, az = np.deg2rad(30.0), np.deg2rad(-90.0)
    eye = WORKSPACE_CENTRE + 1.2 * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    return _jitter_camera(rng, look_at(eye, WORKSPACE_CENTRE), 0.05, 5.0)


def _ego(rng):
    eye = WORKSPACE_CENTRE + np.array([0.0, 0.0, 0.9])     # 0.4 m above the top of the workspace cube
    return _jitter_camera(rng, look_at(eye, WORKSPACE_CENTRE, up=(0.0, 1.0, 0.0)), 0.05, 5.0)


def _side(rng):
    el, az = np.deg2rad(15.0), np.deg2rad(0.0)
    eye = WORKSPACE_CENTRE + 1.6 * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    return _jitter_camera(rng, look_at(eye, WORKSPACE_CENTRE), 0.05, 5.0)


_CAMERA_KINDS = (_third_person, _ego, _side)


def scene_from_lists(name, nodes, env_nodes, env_poses, env_cams, meta=None) -> Scene:
    """Pack per-env python lists into the padded arrays of a Scene."""
    E = len(env_nodes)
    K = max(1, max(len(x) for x in env_nodes))
    C = max(1, max(len(x) for x in env_cams))
    ids = np.full((E, K), -1, np.int32)
    poses = np.zeros((E, K, 3, 4), np.float32)
    poses[:, :, :, :3] = np.eye(3, dtype=np.float32)
    cpe = np.zeros(E, np.int32)
    intr = np.zeros((E, C, 4), np.float32)
    res = np.zeros((E, C, 2), np.int32)
    cpose = np.zeros((E, C, 3, 4), np.float32)
    for e in range(E):
        for j, (k, P) in enumerate(zip(env_nodes[e], env_poses[e])):
            ids[e, j] = k
            poses[e, j] = P
        cpe[e] = len(env_cams[e])
        for c, (fx, fy, cx, cy, w, h, P) in enumerate(env_cams[e]):
            intr[e, c] = (fx, fy, cx, cy)
            res[e, c] = (w, h)
            cpose[e, c] = P
    return Scene(name, nodes, ids, poses, cpe, intr, res, cpose, meta or {})


# ----------------------------------------------------------------------------- workloads
def config1(seed: int = 1, n_bg: int = 8000, n_obj: int = 2000, res: int = 128, f: float = 110.0) -> Scene:
    """1 env x 1 camera 128x128 (f=110, c=64); 8k + 2k Gaussians uniform in [-2,2]^3.

    log-scales N(-3,0.5), uniform rotations, opacity = sigmoid(N(0,1.5)), SH degree 0 with
    colours U[0,1]; the object node sits at a seeded pose (uniform rotation,
    t ~ U[-0.5,0.5]^3).  Camera at (0,0,-5) looking along +z.
    """
    rng = _rng(seed, 1)
    bg = uniform_cube_node(rng, n_bg, 2.0, -3.0, 0.5, 0.0, 1.5, 0, None, "background")
    obj = uniform_cube_node(rng, n_obj, 2.0, -3.0, 0.5, 0.0, 1.5, 0, None, "object")
    P_obj = random_pose(rng, 0.5)
    I = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    cam = np.concatenate([np.eye(3), np.array([[0.0], [0.0], [5.0]])], axis=1)
    c = res / 2.0
    return scene_from_lists("config1", [bg, obj], [[0, 1]], [[I, P_obj]],
                             [[(f, f, c, c, res, res, cam)]], {"seed": seed})


def fd_subset(seed: int = 1, n: int = 200) -> Scene:
    """200 Gaussians of the config-1 law, 32x32 camera with f=27.5, c=16."""
    return config1(seed, n_bg=n - n // 4, n_obj=n // 4, res=32, f=27.5)


def config2(seed: int = 1, n_envs: int = 64, n_bg: int = 1_000_000, n_obj: int = 20_000,
            n_objects: int = 4, width: int = 640, height: int = 480, f: float = 500.0,
            sh_degree: int = 3) -> Scene:
    """64 envs x 2 cameras 640x480; shared 1M-Gaussian room + 4 objects x 20k at per-env poses."""
    rng = _rng(seed, 2)
    nodes = [room_node(rng, n_bg, sh_degree, name="room")]
    nodes += [object_node(rng, n_obj, sh_degree, name=f"object{i}") for i in range(n_objects)]
    I = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    sx, sy = width / 640.0, height / 480.0
    env_nodes, env_poses, env_cams = [], [], []
    for _ in range(n_envs):
        env_nodes.append(list(range(n_objects + 1)))
        env_poses.append([I] + [workspace_pose(rng) for _ in range(n_objects)])
        env_cams.append([(f * sx, f * sy, width / 2.0, height / 2.0, width, height, k(rng))
                         for k in _CAMERA_KINDS[:2]])
    return scene_from_lists("config2", nodes, env_nodes, env_poses, env_cams, {"seed": seed})


_RESOLUTIONS = ((320, 240), (640, 480), (1280, 720))


def config3(seed: int = 1, n_envs: int = 256, n_bg: int = 500_000, n_assets: int = 64,
            asset_lo: int = 5_000, asset_hi: int = 200_000, max_nodes: int = 12,
            resolutions=_RESOLUTIONS, sh_degree: int = 3) -> Scene:
    """256 envs, 1-12 distinct assets each from a pool of 64 (sizes log-uniform 5k-200k),
    1-3 cameras per env at resolutions drawn from {320x240, 640x480, 1280x720}, f = 0.78 W."""
    rng = _rng(seed, 3)
    nodes = [room_node(rng, n_bg, sh_degree, name="room")]
    sizes = np.exp(rng.uniform(math.log(asset_lo), math.log(asset_hi), n_assets)).astype(np.int64)
    nodes += [object_node(rng, int(s), sh_degree, name=f"asset{i}") for i, s in enumerate(sizes)]
    I = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    env_nodes, env_poses, env_cams = [], [], []
    for _ in range(n_envs):
        k = int(rng.integers(1, max_nodes + 1))
        picks = sorted(int(a) + 1 for a in rng.choice(n_assets, size=min(k, n_assets), replace=False))
        env_nodes.append([0] + picks)
        env_poses.append([I] + [workspace_pose(rng) for _ in picks])
        cams = []
        for kind in _CAMERA_KINDS[: int(rng.integers(1, 4))]:
            w, h = resolutions[int(rng.integers(0, len(resolutions)))]
            fw = 0.78 * w
            cams.append((fw, fw, w / 2.0, h / 2.0, w, h, kind(rng)))
        env_cams.append(cams)
    return scene_from_lists("config3", nodes, env_nodes, env_poses, env_cams, {"seed": seed})


def config4(seed: int = 1, n_bg: int = 300_000, n_obj: int = 25_000, n_objects: int = 8,
            res: int = 800, f: float = 700.0, sh_degree: int = 3) -> Scene:
    """Single 800x800 view (f=700, c=400) of a 300k room + 8 objects x 25k: 500k SH-3 Gaussians."""
    rng = _rng(seed, 4)
    nodes = [room_node(rng, n_bg, sh_degree, name="room")]
    nodes += [object_node(rng, n_obj, sh_degree, name=f"object{i}") for i in range(n_objects)]
    I = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    poses = [I] + [workspace_pose(rng) for _ in range(n_objects)]
    s = res / 800.0
    cam = (f * s, f * s, res / 2.0, res / 2.0, res, res, _third_person(rng))
    return scene_from_lists("config4", nodes, [list(range(n_objects + 1))], [poses], [[cam]], {"seed": seed})


def config5(seed: int = 1, n_envs: int = 128, n_bg: int = 3_000_000, n_obj: int = 50_000,
            n_objects: int = 6, width: int = 640, height: int = 480, f: float = 500.0,
            sh_degree: int = 3) -> Scene:
    """128 envs x 3 cameras 640x480; 3M room + 6 objects x 50k (stored BF16/FP16 by the caller)."""
    rng = _rng(seed, 5)
    nodes = [room_node(rng, n_bg, sh_degree, name="room")]
    nodes += [object_node(rng, n_obj, sh_degree, name=f"object{i}") for i in range(n_objects)]
    I = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    sx, sy = width / 640.0, height / 480.0
    env_nodes, env_poses, env_cams = [], [], []
    for _ in range(n_envs):
        env_nodes.append(list(range(n_objects + 1)))
        env_poses.append([I] + [workspace_pose(rng) for _ in range(n_objects)])
        env_cams.append([(f * sx, f * sy, width / 2.0, height / 2.0, width, height, k(rng))
                         for k in _CAMERA_KINDS])
    return scene_from_lists("config5", nodes, env_nodes, env_poses, env_cams, {"seed": seed})


CONFIGS = {"config1": config1, "config2": config2, "config3": config3, "config4": config4,
           "config5": config5, "fd_subset": fd_subset}


def make_config(name: str, seed: int = 1, **kw) -> Scene:
    return CONFIGS[name](seed, **kw)


def select_views(scene: Scene, views) -> Scene:
    """A scene holding only the listed (env, cam) views, each as its own single-camera env."""
    env_nodes, env_poses, env_cams = [], [], []
    for e, c in views:
        ks = [int(k) for k in scene.env_node_ids[e] if k >= 0]
        env_nodes.append(ks)
        env_poses.append([scene.node_poses[e, j] for j in range(len(ks))])
        fx, fy, cx, cy = (float(x) for x in scene.cam_intr[e, c])
        w, h = (int(x) for x in scene.cam_res[e, c])
        env_cams.append([(fx, fy, cx, cy, w, h, scene.cam_pose[e, c])])
    return scene_from_lists(scene.name + "-views", scene.nodes, env_nodes, env_poses, env_cams, dict(scene.meta))


# ------------------------------------------------------------------------ image randomisation
# Per-view parameters of the randomisation applied to rendered frames (Sec. IV: overlay blend,
# HSV jitter, random gamma); the record layout of the C struct dgs_augment.
AUGMENT_DTYPE = np.dtype([("hue_shift", "<f4"), ("sat_scale", "<f4"), ("val_scale", "<f4"), ("gamma", "<f4"),
                          ("overlay_beta", "<f4"), ("overlay_frame", "<i4"), ("overlay_x", "<i4"),
                          ("overlay_y", "<i4")])


def overlay_frames(seed: int = 1, n_frames: int = 8, width: int = 1280, height: int = 720) -> np.ndarray:
    """A seeded synthetic stand-in for the Internet video clips whose crops the paper blends
    into rendered frames: uint8 [n_frames, height, width, 3].  Each frame is a smooth colour
    field (a few drifting plane waves per channel) with a dozen flat-coloured discs and boxes
    moving at constant velocity across the clip, plus mild per-pixel noise, so that crops hold
    edges, flat regions and gradients as video does."""
    rng = _rng(seed, 101)
    y, x = np.mgrid[0:height, 0:width].astype(np.float64)
    waves = rng.uniform(-1.0, 1.0, size=(3, 4, 2)) * (2 * math.pi / np.array([width, height]) * 3.0)
    phase0 = rng.uniform(0, 2 * math.pi, size=(3, 4))
    drift = rng.uniform(-0.3, 0.3, size=(3, 4))
    n_shapes = 12
    kind = rng.integers(0, 2, size=n_shapes)
    c0 = rng.uniform([0, 0], [width, height], size=(n_shapes, 2))
    vel = rng.uniform(-12.0, 12.0, size=(n_shapes, 2))
    size = rng.uniform(0.03, 0.15, size=n_shapes) * min(width, height)
    colour = rng.uniform(0.0, 1.0, size=(n_shapes, 3))
    frames = np.empty((n_frames, height, width, 3), dtype=np.uint8)
    for f in range(n_frames):
        img = np.empty((height, width, 3))
        for ch in range(3):
            acc = np.zeros((height, width))
            for k in range(4):
                acc += np.cos(waves[ch, k, 0] * x + waves[ch, k, 1] * y + phase0[ch, k] + drift[ch, k] * f)
            img[..., ch] = 0.5 + 0.12 * acc
        for s in range(n_shapes):
            cx, cy = c0[s] + vel[s] * f
            if kind[s] == 0:
                m = (x - cx) ** 2 + (y - cy) ** 2 <= size[s] ** 2
            else:
                m = (np.abs(x - cx) <= size[s]) & (np.abs(y - cy) <= 0.6 * size[s])
            img[m] = colour[s]
        img += rng.normal(0.0, 0.02, size=img.shape)
        frames[f] = np.clip(np.rint(img * 255.0), 0, 255).astype(np.uint8)
    return frames


def augment_params(seed: int, n_views: int, n_frames: int, overlay_w: int, overlay_h: int,
                   hue: float = 0.05, sat=(0.7, 1.3), val=(0.7, 1.3), gamma=(0.7, 1.5), beta=(0.1, 0.4),
                   p_overlay: float = 0.5) -> np.ndarray:
    """Seeded per-view randomisation parameters (AUGMENT_DTYPE [n_views]): hue shift uniform in
    [-hue, hue] turns, saturation and value scales and gamma uniform in their ranges, and with
    probability p_overlay an overlay weight uniform in `beta` (else 0) with a uniformly drawn
    frame and crop origin."""
    rng = _rng(seed, 102)
    p = np.zeros(n_views, dtype=AUGMENT_DTYPE)
    p["hue_shift"] = rng.uniform(-hue, hue, n_views)
    p["sat_scale"] = rng.uniform(*sat, n_views)
    p["val_scale"] = rng.uniform(*val, n_views)
    p["gamma"] = rng.uniform(*gamma, n_views)
    on = rng.uniform(size=n_views) < p_overlay
    p["overlay_beta"] = np.where(on, rng.uniform(*beta, n_views), 0.0)
    p["overlay_frame"] = rng.integers(0, n_frames, n_views)
    p["overlay_x"] = rng.integers(0, overlay_w, n_views)
    p["overlay_y"] = rng.integers(0, overlay_h, n_views)
    return p


# ------------------------------------------------------------------------------------- LiDAR
def lidar_pattern(channels: int = 32, azimuths: int = 1024, el_min_deg: float = -30.67,
                  el_max_deg: float = 10.67, az0_deg: float = 0.0, az_span_deg: float = 360.0,
                  tile=(4, 8)) -> np.ndarray:
    """Beam directions of a spinning multi-channel LiDAR in its own frame (x forward, y left,
    z up): `channels` elevations spaced evenly over [el_min, el_max] (the defaults are those
    of a 32-beam automotive unit) times `azimuths` evenly spaced azimuths; float32 [channels *
    azimuths, 3] unit vectors.  Order: tiles of tile[0] channels x tile[1] azimuths (each tile
    channel-major, tiles channel-block-major), so that every 32 consecutive beams are
    neighbours; tile=None gives plain channel-major order."""
    el = np.deg2rad(np.linspace(el_min_deg, el_max_deg, channels))
    az = np.deg2rad(az0_deg + az_span_deg * np.arange(azimuths) / azimuths)
    ce, se = np.cos(el)[:, None], np.sin(el)[:, None]
    d = np.stack([ce * np.cos(az)[None, :], ce * np.sin(az)[None, :], np.broadcast_to(se, (channels, azimuths))],
                 axis=-1)
    if tile is not None:
        c, a = np.meshgrid(np.arange(channels), np.arange(azimuths), indexing="ij")
        tc, ta = tile
        order = np.lexsort(((a % ta).ravel(), (c % tc).ravel(), (a // ta).ravel(), (c // tc).ravel()))
        return np.ascontiguousarray(d.reshape(-1, 3)[order].astype(np.float32))
    return np.ascontiguousarray(d.reshape(-1, 3).astype(np.float32))


def lidar_sensors(seed: int, n_envs: int, radius=(1.0, 2.0), height=(0.8, 1.6), tilt_deg: float = 2.0):
    """One LiDAR per env, mounted as on a mobile robot near the workspace: at a distance in
    `radius` from the workspace centre (horizontally), at a height in `height`, facing the
    workspace within 30 degrees of yaw, tilted by N(0, tilt_deg).  Returns (sensor_env int32
    [n_envs], world_from_sensor float32 [n_envs, 3, 4])."""
    rng = _rng(seed, 103)
    poses = np.zeros((n_envs, 3, 4), np.float64)
    for e in range(n_envs):
        phi = rng.uniform(-np.pi, np.pi)
        r = rng.uniform(*radius)
        p = np.array([WORKSPACE_CENTRE[0] + r * math.cos(phi), WORKSPACE_CENTRE[1] + r * math.sin(phi),
                      rng.uniform(*height)])
        yaw = phi + np.pi + rng.uniform(-np.pi / 6, np.pi / 6)      # x axis towards the workspace
        ax = rng.normal(size=2)
        R = _rot_axis([ax[0], ax[1], 0.0], np.deg2rad(rng.normal(0.0, tilt_deg))) @ _rot_axis([0, 0, 1], yaw)
        poses[e] = np.concatenate([_orthonormalise(R), p[:, None]], axis=1)
    return np.arange(n_envs, dtype=np.int32), poses.astype(np.float32)


# ------------------------------------------------------------------------------------ meshes
def mesh_icosphere(subdiv: int = 3, radius: float = 0.05):
    """A closed triangle mesh of a sphere (icosahedron subdivided `subdiv` times, vertices pushed
    to the sphere), outward winding: (vertices float32 [V,3], faces int32 [F,3]), F = 20 * 4^subdiv."""
    t = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
         (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]
        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return (np.asarray(verts) * radius).astype(np.float32), np.asarray(faces, np.int32)


def mesh_heightfield(seed: int, nx: int, ny: int, size: float = 1.0, amp: float = 0.05):
    """A noisy terrain-like sheet: an nx x ny vertex grid over [0, size]^2 with heights from a few
    random plane waves, two triangles per cell (upward normals), and per-vertex colours from
    another smooth field: (vertices float32 [V,3], faces int32 [F,3], colours float32 [V,3]),
    F = 2 (nx - 1)(ny - 1)."""
    rng = _rng(seed, 104)
    xs, ys = np.meshgrid(np.linspace(0, size, nx), np.linspace(0, size, ny), indexing="xy")
    k = rng.uniform(-12, 12, (5, 2)) / size
    ph = rng.uniform(0, 2 * np.pi, 5)
    z = amp * sum(np.sin(k[i, 0] * xs + k[i, 1] * ys + ph[i]) for i in range(5)) / 5.0
    z += rng.normal(0.0, amp * 0.05, z.shape)
    verts = np.stack([xs, ys, z], axis=-1).reshape(-1, 3)
    idx = np.arange(nx * ny).reshape(ny, nx)
    a, b, c, d = idx[:-1, :-1].ravel(), idx[:-1, 1:].ravel(), idx[1:, :-1].ravel(), idx[1:, 1:].ravel()
    faces = np.concatenate([np.stack([a, b, d], 1), np.stack([a, d, c], 1)], axis=0)
    col = 0.5 + 0.4 * np.stack([np.sin(3 * xs + ph[0]), np.sin(4 * ys + ph[1]), np.cos(2 * (xs + ys) + ph[2])],
                               axis=-1).reshape(-1, 3)
    return verts.astype(np.float32), faces.astype(np.int32), col.astype(np.float32)


# ------------------------------------------------------------------------------- depth views
def sphere_depth_views(centre, radius: float, n_views: int = 8, width: int = 96, height: int = 72,
                       f: float = 80.0, dist: float = 1.0, seed: int = 0):
    """Synthetic depth maps of a sphere for fusion tests: n_views pinhole cameras on a ring at
    `dist` from the centre (random elevation in +-30 degrees) looking at it; per view the
    camera-space z of the first ray-sphere intersection through each pixel centre (0 where the
    ray misses) and coverage 1 / 0.  Returns (cams [(fx, fy, cx, cy, W, H, cam_from_world)],
    depth float32 [V, H, W], alpha float32 [V, H, W])."""
    rng = _rng(seed, 105)
    c = np.asarray(centre, np.float64)
    cams, depth, alpha = [], [], []
    for k in range(n_views):
        az = 2 * np.pi * k / n_views + rng.uniform(-0.2, 0.2)
        el = rng.uniform(-np.pi / 6, np.pi / 6)
        eye = c + dist * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        P = look_at(eye, c)
        R, t = P[:, :3], P[:, 3]
        ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
        dc = np.stack([(xs + 0.5 - width / 2) / f, (ys + 0.5 - height / 2) / f, np.ones_like(xs)], axis=-1)
        dw = dc @ R                                  # world direction (unnormalised, camera z = 1)
        oc = eye - c
        a = np.sum(dw * dw, axis=-1)
        b = 2 * dw @ oc
        cc = oc @ oc - radius * radius
        disc = b * b - 4 * a * cc
        hit = disc >= 0
        s = np.where(hit, (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a), 0.0)   # s = camera-space z
        hit &= s > 0
        depth.append(np.where(hit, s, 0.0).astype(np.float32))
        alpha.append(hit.astype(np.float32))
        cams.append((f, f, width / 2.0, height / 2.0, width, height, P.astype(np.float32)))
    return cams, np.stack(depth), np.stack(alpha)
