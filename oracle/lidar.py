"""ctypes front end of the FP64 LiDAR oracle (lidar.cpp).  Test infrastructure only.

Traces rays (sensor, direction) through the Gaussians of the sensor's env by brute force and
returns per ray the unnormalised range D = sum w t*, the opacity A = 1 - T, and the FP32
tolerance the oracle derives for each (see lidar.cpp).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import oracle as _o


class _LScene(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("node_n", C.c_void_p), ("mean", C.c_void_p), ("log_scale", C.c_void_p),
                ("quat", C.c_void_p), ("opacity_logit", C.c_void_p), ("E", C.c_int32), ("K", C.c_int32),
                ("env_node_ids", C.c_void_p), ("node_poses", C.c_void_p)]


class _LOpts(C.Structure):
    _fields_ = [("alpha_min", C.c_double), ("alpha_max", C.c_double), ("t_min", C.c_double), ("q_max", C.c_double),
                ("r_min", C.c_double), ("r_max", C.c_double), ("eps_rel", C.c_double), ("nthreads", C.c_int32)]


@dataclass
class LidarOptions:
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    q_max: float = 9.0
    r_min: float = 0.05
    r_max: float = 30.0
    eps_rel: float = 1e-7
    nthreads: int = 0


@dataclass
class LidarResult:
    d: np.ndarray          # [S, J] unnormalised range sum w t*
    a: np.ndarray          # [S, J] opacity 1 - T
    tol_d: np.ndarray
    tol_a: np.ndarray
    n_comp: np.ndarray     # hits composited
    n_amb: np.ndarray      # ambiguous decisions met


_fn = None


def _lib():
    global _fn
    if _fn is None:
        lib = _o._load()
        lib.oracle_lidar_rays.restype = C.c_int
        lib.oracle_lidar_rays.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                          C.c_void_p] + [C.c_void_p] * 6
        _fn = lib.oracle_lidar_rays
    return _fn


def trace(scene, sensor_env, sensor_pose, dirs, opts: LidarOptions | None = None, packed=None) -> LidarResult:
    """Sec. III-C: LiDAR returns by ray tracing the env's Gaussians (definition in lidar.cpp).
    sensor_env [S] int, sensor_pose [S,3,4] world_from_sensor, dirs [J,3] sensor-frame
    directions (normalised inside)."""
    opts = opts or LidarOptions()
    pk = packed or _o._Packed(scene)
    ls = _LScene()
    ls.n_nodes = len(scene.nodes)
    ls.node_n, ls.mean, ls.log_scale = pk.node_n.ctypes.data, pk.mean.ctypes.data, pk.log_scale.ctypes.data
    ls.quat, ls.opacity_logit = pk.quat.ctypes.data, pk.opacity_logit.ctypes.data
    ls.E, ls.K = pk.env_node_ids.shape
    ls.env_node_ids, ls.node_poses = pk.env_node_ids.ctypes.data, pk.node_poses.ctypes.data
    lo = _LOpts(*(float(getattr(opts, k)) for k in ("alpha_min", "alpha_max", "t_min", "q_max", "r_min", "r_max",
                                                     "eps_rel")), int(opts.nthreads))
    se = np.ascontiguousarray(sensor_env, np.int32)
    sp = np.ascontiguousarray(np.asarray(sensor_pose, np.float64).reshape(-1, 12))
    dr = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 3))
    S, J = len(se), len(dr)
    out = [np.zeros((S, J), np.float64) for _ in range(4)]
    nc = np.zeros((S, J), np.int32)
    na = np.zeros((S, J), np.int32)
    rc = _lib()(C.byref(ls), C.byref(lo), S, se.ctypes.data, sp.ctypes.data, J, dr.ctypes.data,
                *(x.ctypes.data for x in out), nc.ctypes.data, na.ctypes.data)
    assert rc == 0
    return LidarResult(out[0], out[1], out[2], out[3], nc, na)
