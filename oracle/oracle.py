"""ctypes front end of the FP64 oracle (oracle.cpp).  Test infrastructure only."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_SRCS = [_SRC, os.path.join(_HERE, "lidar.cpp")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile oracle.cpp and lidar.cpp into liboracle.so next to them (g++, -O2, portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(p) for p in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, *_SRCS])
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("node_n", C.c_void_p), ("node_deg", C.c_void_p),
                ("mean", C.c_void_p), ("log_scale", C.c_void_p), ("quat", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p),
                ("E", C.c_int32), ("K", C.c_int32), ("C", C.c_int32),
                ("env_node_ids", C.c_void_p), ("node_poses", C.c_void_p), ("cams_per_env", C.c_void_p),
                ("cam_intr", C.c_void_p), ("cam_res", C.c_void_p), ("cam_pose", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("z_near", C.c_double), ("lowpass", C.c_double), ("alpha_min", C.c_double),
                ("alpha_max", C.c_double), ("t_min", C.c_double), ("q_max", C.c_double),
                ("guard", C.c_double), ("bg", C.c_double * 3), ("eps_rel", C.c_double),
                ("max_flips", C.c_int32), ("nthreads", C.c_int32),
                ("bruteforce", C.c_int32), ("max_branches", C.c_int32)]


@dataclass
class OracleOptions:
    z_near: float = 0.01
    lowpass: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    q_max: float = 9.0
    guard: float = 1.3
    bg: tuple = (0.0, 0.0, 0.0)
    eps_rel: float = 1e-7
    max_flips: int = 4
    nthreads: int = 0
    bruteforce: int = 0
    max_branches: int = 64

    def _c(self) -> _Opts:
        o = _Opts()
        for k in ("z_near", "lowpass", "alpha_min", "alpha_max", "t_min", "q_max", "guard",
                  "eps_rel"):
            setattr(o, k, float(getattr(self, k)))
        o.bg = (C.c_double * 3)(*[float(b) for b in self.bg])
        o.max_flips, o.nthreads, o.bruteforce = int(self.max_flips), int(self.nthreads), int(self.bruteforce)
        o.max_branches = int(self.max_branches)
        return o


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            lib.oracle_project_view.restype = C.c_int64
            lib.oracle_project_view.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int64]
            lib.oracle_render_view.restype = C.c_int
            lib.oracle_render_view.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 8 + \
                [C.c_int64, C.c_void_p, C.c_void_p]
            lib.oracle_backward_view.restype = C.c_int
            lib.oracle_backward_view.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 14
            lib.oracle_sh_basis.restype = None
            lib.oracle_sh_basis.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            _lib = lib
    return _lib


class _Packed:
    """FP64 copies of a scene's arrays, kept alive while the C structure points at them."""

    def __init__(self, scene, attr_override=None):
        nodes = scene.nodes
        f8 = np.float64
        self.node_n = np.array([nd.n for nd in nodes], np.int64)
        self.node_deg = np.array([nd.sh_degree for nd in nodes], np.int32)
        G = int(self.node_n.sum())
        get = attr_override or (lambda nd, name: getattr(nd, name))
        self.mean = np.ascontiguousarray(np.concatenate([get(nd, "mean") for nd in nodes]).astype(f8).reshape(G, 3))
        self.log_scale = np.ascontiguousarray(np.concatenate([get(nd, "log_scale") for nd in nodes]).astype(f8).reshape(G, 3))
        self.quat = np.ascontiguousarray(np.concatenate([get(nd, "quat") for nd in nodes]).astype(f8).reshape(G, 4))
        self.opacity_logit = np.ascontiguousarray(np.concatenate([get(nd, "opacity_logit") for nd in nodes]).astype(f8).reshape(G))
        sh = np.zeros((G, 16, 3), f8)
        off = 0
        for nd in nodes:
            s = np.asarray(get(nd, "sh"), f8).reshape(nd.n, (nd.sh_degree + 1) ** 2, 3)
            sh[off:off + nd.n, : s.shape[1]] = s
            off += nd.n
        self.sh = sh
        self.env_node_ids = np.ascontiguousarray(scene.env_node_ids, np.int32)
        self.node_poses = np.ascontiguousarray(np.asarray(scene.node_poses, f8).reshape(scene.env_node_ids.shape + (12,)))
        self.cams_per_env = np.ascontiguousarray(scene.cams_per_env, np.int32)
        self.cam_intr = np.ascontiguousarray(scene.cam_intr, f8)
        self.cam_res = np.ascontiguousarray(scene.cam_res, np.int32)
        self.cam_pose = np.ascontiguousarray(np.asarray(scene.cam_pose, f8).reshape(scene.cam_res.shape[:2] + (12,)))
        s = _Scene()
        s.n_nodes = len(nodes)
        s.node_n, s.node_deg = self.node_n.ctypes.data, self.node_deg.ctypes.data
        s.mean, s.log_scale, s.quat = self.mean.ctypes.data, self.log_scale.ctypes.data, self.quat.ctypes.data
        s.opacity_logit, s.sh = self.opacity_logit.ctypes.data, self.sh.ctypes.data
        s.E, s.K = self.env_node_ids.shape
        s.C = self.cam_res.shape[1]
        s.env_node_ids, s.node_poses = self.env_node_ids.ctypes.data, self.node_poses.ctypes.data
        s.cams_per_env, s.cam_intr = self.cams_per_env.ctypes.data, self.cam_intr.ctypes.data
        s.cam_res, s.cam_pose = self.cam_res.ctypes.data, self.cam_pose.ctypes.data
        self.c = s
        self.G = G


def _p(a):
    return None if a is None else a.ctypes.data


def project_view(scene, e: int, c: int, opts: OracleOptions | None = None, packed=None) -> np.ndarray:
    """Sec. III-A (EWA splatting, SH colour, depth).  Per-instance projection of view (e, c):
    columns gid, u, v, z, conic a, b, c, cov xx, xy, yy, opacity, r, g, b, present, near_ambiguous
    (instances behind the near plane are listed only when that decision is ambiguous)."""
    lib = _load()
    pk = packed or _Packed(scene)
    o = (opts or OracleOptions())._c()
    cap = pk.G
    out = np.zeros((cap, 16), np.float64)
    n = lib.oracle_project_view(C.byref(pk.c), C.byref(o), e, c, _p(out), cap)
    if n < 0:
        raise ValueError("bad view")
    return out[:n]


@dataclass
class ViewResult:
    rgb: np.ndarray
    depth: np.ndarray
    alpha: np.ndarray
    tol_rgb: np.ndarray
    tol_d: np.ndarray
    n_alt: np.ndarray
    alt: np.ndarray           # [n_alt_total, 6] (r, g, b, d, a, FP32 error bound of a) in pixel order
    ambiguous_pixels: int
    decision_hash: int
    instances: int
    ambiguous_by_kind: dict = field(default=None)
    work: dict = field(default=None)
    grad_amb: np.ndarray = field(default=None)   # pixels with a gradient switch inside its FP32 band
    err_a: np.ndarray = field(default=None)      # FP32 error bound of the primary branch's coverage
    widened_pixels: int = 0                      # pixels whose tolerance covers unexplored flips
    alt_offsets: np.ndarray = field(default=None)

    def alternatives(self, p: int) -> np.ndarray:
        if self.alt_offsets is None:
            self.alt_offsets = np.concatenate([[0], np.cumsum(self.n_alt.reshape(-1))])
        return self.alt[self.alt_offsets[p]: self.alt_offsets[p + 1]]


def render_view(scene, e: int, c: int, opts: OracleOptions | None = None, packed=None) -> ViewResult:
    """Sec. III-A and III-C: RGB, unnormalised depth and coverage of view (e, c) by the plain
    per-pixel definition in oracle.cpp (FP64, depth order by FP64 z), with the FP32-ambiguous
    decisions -- near plane, ellipse, alpha_min, t_min and depth order -- flagged and their
    alternative branches (r, g, b, d, a, error bound of a) returned."""
    lib = _load()
    pk = packed or _Packed(scene)
    o = (opts or OracleOptions())._c()
    W, H = (int(x) for x in scene.cam_res[e, c])
    rgb = np.zeros((H, W, 3)); depth = np.zeros((H, W)); alpha = np.zeros((H, W))
    ea = np.zeros((H, W))
    tr = np.zeros((H, W)); td = np.zeros((H, W)); na = np.zeros((H, W), np.int32)
    ga = np.zeros((H, W), np.int32)
    stats = np.zeros(13, np.int64)
    cap = max(1024, W * H // 8)
    alt = np.zeros((cap, 6))
    args = lambda: (C.byref(pk.c), C.byref(o), e, c, _p(rgb), _p(depth), _p(alpha), _p(ea), _p(tr), _p(td), _p(na),
                    _p(alt), cap, _p(stats), _p(ga))
    rc = lib.oracle_render_view(*args())
    if rc == 1:
        cap = int(stats[0])
        alt = np.zeros((cap, 6))
        rc = lib.oracle_render_view(*args())
    if rc != 0:
        raise ValueError(f"oracle_render_view failed ({rc})")
    kinds = dict(zip(("near", "ellipse", "alpha", "transmittance", "order"),
                     (int(x) for x in (*stats[4:8], stats[11]))))
    work = dict(contributions=int(stats[8]), reached=int(stats[9]), terminated_pixels=int(stats[10]))
    return ViewResult(rgb, depth, alpha, tr, td, na, alt[: int(stats[0])], int(stats[1]),
                      int(np.uint64(stats[2].view(np.uint64))), int(stats[3]), kinds, work, ga.astype(bool),
                      ea, int(stats[12]))


def _grad_buffers(pk, scene, with_error=False):
    E, K = scene.env_node_ids.shape
    g = dict(mean=np.zeros((pk.G, 3)), log_scale=np.zeros((pk.G, 3)), quat=np.zeros((pk.G, 4)),
             opacity_logit=np.zeros(pk.G), sh=np.zeros((pk.G, 16, 3)), pose=np.zeros((E, K, 3, 4)))
    if with_error:
        g.update({"err_" + k: np.zeros_like(v) for k, v in list(g.items())})
    return g


def backward_view(scene, e: int, c: int, grad_rgb, grad_depth=None, opts: OracleOptions | None = None,
                  packed=None, out=None, with_error: bool = False) -> dict:
    """Sec. IV (assets fitted by gradient descent on rendered images).  Adjoint of view (e, c)
    for L = sum(grad_rgb * RGB) + sum(grad_depth * D).

    Returns (or accumulates into `out`) gradients laid out as concatenated node arrays: mean [G,3],
    log_scale [G,3], quat [G,4], opacity_logit [G], sh [G,16,3], pose [E,K,3,4].  with_error adds
    "err_<name>" arrays of the same layouts: the FP32 error model of each gradient entry (header
    of oracle_backward_view in oracle.cpp)."""
    lib = _load()
    pk = packed or _Packed(scene)
    o = (opts or OracleOptions())._c()
    g = out if out is not None else _grad_buffers(pk, scene, with_error)
    gr = np.ascontiguousarray(grad_rgb, np.float64)
    gd = None if grad_depth is None else np.ascontiguousarray(grad_depth, np.float64)
    names = ("mean", "log_scale", "quat", "opacity_logit", "sh", "pose")
    errs = [_p(g["err_" + n]) for n in names] if with_error else [None] * 6
    rc = lib.oracle_backward_view(C.byref(pk.c), C.byref(o), e, c, _p(gr), _p(gd), *[_p(g[n]) for n in names], *errs)
    if rc != 0:
        raise ValueError(f"oracle_backward_view failed ({rc})")
    return g


def backward_scene(scene, grad_rgb_views, grad_depth_views, opts=None, with_error: bool = False) -> dict:
    """Sec. IV: sum of backward_view over all views (lists of per-view gradient images)."""
    pk = _Packed(scene)
    g = _grad_buffers(pk, scene, with_error)
    for v, (e, c) in enumerate(scene.views):
        backward_view(scene, e, c, grad_rgb_views[v], None if grad_depth_views is None else grad_depth_views[v],
                      opts, pk, g, with_error)
    return g


def pose_twist_grad(pose: np.ndarray, grad_pose: np.ndarray) -> np.ndarray:
    """Sec. III-B (rigid node poses): se(3) gradient (rho, phi) of a left perturbation exp(xi^) [R|t]
    from the 3x4 gradient.

    With R' = (I + [phi]x) R and t' = (I + [phi]x) t + rho:  dL/drho = G_t and dL/dphi is the axial
    vector of the skew part of A = G_R R^T + G_t t^T, i.e. (A32-A23, A13-A31, A21-A12)."""
    P = np.asarray(pose, np.float64).reshape(3, 4)
    Gm = np.asarray(grad_pose, np.float64).reshape(3, 4)
    A = Gm[:, :3] @ P[:, :3].T + np.outer(Gm[:, 3], P[:, 3])
    phi = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
    return np.concatenate([Gm[:, 3], phi])


def sh_basis(deg: int, d) -> tuple:
    """Sec. III-A (spherical-harmonics colour): (Y[16], dY[16,3]) of the oracle's real SH basis at
    direction d (entries above deg are 0)."""
    lib = _load()
    dd = np.ascontiguousarray(d, np.float64)
    Y = np.zeros(16); dY = np.zeros((16, 3))
    lib.oracle_sh_basis(int(deg), _p(dd), _p(Y), _p(dY))
    return Y, dY
