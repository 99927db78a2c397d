"""ctypes binding of libdgs (include/dgs.h): the same names, argument marshalling only.

Every step of rendering runs in the CUDA library; this module only converts Python values to
the C structures and calls the exported functions.  It raises if libdgs.so cannot be loaded:
there is no fallback implementation.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgs.so")
DEBUG_LIB_PATH = os.path.join(HERE, "libdgs_debug.so")   # -DDGS_DEBUG: device bounds checks

DGS_OK, DGS_ERR_INVALID_ARG, DGS_ERR_CUDA, DGS_ERR_OOM, DGS_ERR_CAPACITY, DGS_ERR_TIMEOUT, DGS_ERR_UNSUPPORTED = range(7)
DGS_F32, DGS_BF16, DGS_F16 = 0, 1, 2
DGS_MODE_PLAIN, DGS_MODE_BATCHED, DGS_MODE_GRAPH = 0, 1, 2
DGS_PATH_EAGER, DGS_PATH_GRAPH, DGS_PATH_CAPTURED, DGS_PATH_REGROWN, DGS_PATH_KEPT_LISTS = 0, 1, 2, 3, 4
DGS_TUNE_MAX = 16
KERNEL_CLASSES = ("setup", "count", "scan", "emit", "sort", "ranges", "composite", "backward", "graph", "augment",
                  "lidar", "mesh", "tsdf", "backward_project")
STATUS_NAMES = {0: "DGS_OK", 1: "DGS_ERR_INVALID_ARG", 2: "DGS_ERR_CUDA", 3: "DGS_ERR_OOM", 4: "DGS_ERR_CAPACITY",
                5: "DGS_ERR_TIMEOUT", 6: "DGS_ERR_UNSUPPORTED"}


class dgs_node(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("log_scale", C.c_void_p), ("quat", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64),
                ("sh_degree", C.c_int32), ("dtype", C.c_int32)]


class dgs_camera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32), ("cam_from_world", C.c_float * 12)]


class dgs_options(C.Structure):
    _fields_ = [("mode", C.c_int32), ("tile_w", C.c_int32), ("tile_h", C.c_int32), ("exact_tile_test", C.c_int32),
                ("z_near", C.c_float), ("lowpass", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("t_min", C.c_float), ("q_max", C.c_float), ("guard", C.c_float), ("bg", C.c_float * 3),
                ("profile", C.c_int32), ("views_per_group", C.c_int32), ("spin_limit_us", C.c_int32),
                ("check_binning", C.c_int32), ("test_fault", C.c_int32), ("keep_lists", C.c_int32)]


class dgs_node_grads(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("log_scale", C.c_void_p), ("quat", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p)]


class dgs_stats(C.Structure):
    _fields_ = [("n_views", C.c_int64), ("n_pixels", C.c_int64), ("n_instances", C.c_int64),
                ("n_visible", C.c_int64), ("n_pairs", C.c_int64), ("n_groups", C.c_int32), ("key_bits", C.c_int32),
                ("px_evaluated", C.c_int64), ("px_reached", C.c_int64), ("px_composited", C.c_int64),
                ("path", C.c_int32), ("graph_captures", C.c_int32), ("bwd_reductions", C.c_int64)]


class dgs_tune_result(C.Structure):
    _fields_ = [("n", C.c_int32), ("best", C.c_int32), ("tile_w", C.c_int32 * DGS_TUNE_MAX),
                ("tile_h", C.c_int32 * DGS_TUNE_MAX), ("ms", C.c_float * DGS_TUNE_MAX)]


class dgs_augment(C.Structure):
    _fields_ = [("hue_shift", C.c_float), ("sat_scale", C.c_float), ("val_scale", C.c_float), ("gamma", C.c_float),
                ("overlay_beta", C.c_float), ("overlay_frame", C.c_int32), ("overlay_x", C.c_int32),
                ("overlay_y", C.c_int32)]


class dgs_lidar(C.Structure):
    _fields_ = [("env", C.c_int32), ("world_from_sensor", C.c_float * 12)]


EXPORTED = ("dgs_default_options", "dgs_context_create", "dgs_context_destroy", "dgs_last_error",
            "dgs_workspace_query", "dgs_render", "dgs_last_stats", "dgs_kernel_times", "dgs_last_launches",
            "dgs_render_noalloc", "dgs_render_backward", "dgs_autotune", "dgs_spatial_order",
            "dgs_set_augment", "dgs_augment_rgb", "dgs_lidar_build", "dgs_lidar_trace", "dgs_mesh_to_gaussians",
            "dgs_tsdf_integrate", "dgs_pose_twist_grad", "dgs_set_options", "dgs_workspace_query_batch",
            "dgs_build_flags")
DGS_BUILD_DEBUG = 1

_lib = None
_lock = threading.Lock()


class DgsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def load(path: str | None = None) -> C.CDLL:
    """Loads libdgs.so (built in-tree by build.py).  Raises if it is missing.  With a path (for
    instance DEBUG_LIB_PATH) that library is loaded and returned without replacing the default."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libdgs.so not found at {p}: build it with paper_2507_21981_gb300.build.build()")
        lib = C.CDLL(p)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        lib.dgs_default_options.restype = None
        lib.dgs_default_options.argtypes = [C.POINTER(dgs_options)]
        lib.dgs_context_create.restype = C.c_int
        lib.dgs_context_create.argtypes = [C.POINTER(vp), C.POINTER(dgs_options)]
        lib.dgs_context_destroy.restype = C.c_int
        lib.dgs_context_destroy.argtypes = [vp]
        lib.dgs_last_error.restype = C.c_char_p
        lib.dgs_last_error.argtypes = [vp]
        lib.dgs_workspace_query.restype = C.c_int
        lib.dgs_workspace_query.argtypes = [vp, C.POINTER(C.c_size_t)]
        lib.dgs_render.restype = C.c_int
        lib.dgs_render.argtypes = [vp, C.POINTER(dgs_node), i32, vp, i32, i32, vp, C.POINTER(dgs_camera), vp, i32,
                                   vp, vp, vp, vp, vp]
        lib.dgs_last_stats.restype = C.c_int
        lib.dgs_last_stats.argtypes = [vp, C.POINTER(dgs_stats)]
        lib.dgs_kernel_times.restype = C.c_int
        lib.dgs_kernel_times.argtypes = [vp, C.POINTER(C.c_float)]
        lib.dgs_last_launches.restype = C.c_int64
        lib.dgs_last_launches.argtypes = [vp]
        lib.dgs_build_flags.restype = C.c_int32
        lib.dgs_build_flags.argtypes = []
        lib.dgs_render_backward.restype = C.c_int
        lib.dgs_render_backward.argtypes = [vp, C.POINTER(dgs_node), i32, vp, i32, i32, vp, C.POINTER(dgs_camera), vp,
                                            i32, vp, vp, vp, vp, C.POINTER(dgs_node_grads), vp, vp, vp]
        lib.dgs_spatial_order.restype = C.c_int
        lib.dgs_spatial_order.argtypes = [vp, i64, vp]
        lib.dgs_autotune.restype = C.c_int
        lib.dgs_autotune.argtypes = [vp, C.POINTER(dgs_node), i32, vp, i32, i32, vp, C.POINTER(dgs_camera), vp, i32,
                                     vp, vp, vp, vp, vp, i32, i32, C.POINTER(dgs_tune_result), vp]
        lib.dgs_render_noalloc.restype = C.c_int
        lib.dgs_render_noalloc.argtypes = [C.POINTER(dgs_options), C.POINTER(dgs_node), i32, vp, i32, i32, vp,
                                           C.POINTER(dgs_camera), vp, i32, vp, vp, vp, vp, vp]
        lib.dgs_set_augment.restype = C.c_int
        lib.dgs_set_augment.argtypes = [vp, vp, i32, vp, i32, i32, i32]
        lib.dgs_augment_rgb.restype = C.c_int
        lib.dgs_augment_rgb.argtypes = [vp, vp, vp, vp, i32, vp]
        lib.dgs_lidar_build.restype = C.c_int
        lib.dgs_lidar_build.argtypes = [vp, C.POINTER(dgs_node), i32, vp]
        lib.dgs_lidar_trace.restype = C.c_int
        lib.dgs_lidar_trace.argtypes = [vp, C.POINTER(dgs_node), i32, vp, i32, i32, vp, C.POINTER(dgs_lidar), i32, vp,
                                        i32, C.c_float, C.c_float, vp, vp, vp]
        lib.dgs_mesh_to_gaussians.restype = C.c_int
        lib.dgs_mesh_to_gaussians.argtypes = [vp, vp, i64, vp, i64, vp, C.c_float, C.c_float, i32, vp, vp, vp, vp, vp,
                                              vp]
        lib.dgs_tsdf_integrate.restype = C.c_int
        lib.dgs_pose_twist_grad.argtypes = [vp, vp, i64, vp, vp]
        lib.dgs_set_options.argtypes = [vp, C.POINTER(dgs_options)]
        lib.dgs_workspace_query_batch.argtypes = [vp, C.POINTER(dgs_node), i32, vp, i32, i32, vp,
                                                  C.POINTER(dgs_camera), vp, i32, vp, C.POINTER(C.c_size_t), vp]
        lib.dgs_workspace_query_batch.restype = C.c_int
        lib.dgs_set_options.restype = C.c_int
        lib.dgs_pose_twist_grad.restype = C.c_int
        lib.dgs_tsdf_integrate.argtypes = [vp, vp, vp, i32, i32, i32, vp, C.c_float, C.c_float, C.c_float, C.c_float,
                                           C.POINTER(dgs_camera), i32, vp, vp, vp, vp]
        if path is None:
            _lib = lib
        return lib


# ----------------------------------------------------------------------------- same-name wrappers
def dgs_default_options() -> dgs_options:
    o = dgs_options()
    load().dgs_default_options(C.byref(o))
    return o


def dgs_context_create(opt: dgs_options | None = None) -> C.c_void_p:
    h = C.c_void_p()
    rc = load().dgs_context_create(C.byref(h), C.byref(opt) if opt is not None else None)
    if rc != DGS_OK:
        raise DgsError(rc, "dgs_context_create")
    return h


def dgs_set_options(ctx, opt: dgs_options) -> int:
    return load().dgs_set_options(ctx, C.byref(opt))


def dgs_context_destroy(ctx) -> int:
    return load().dgs_context_destroy(ctx)


def dgs_last_error(ctx) -> str:
    s = load().dgs_last_error(ctx)
    return s.decode() if s else ""


def dgs_workspace_query(ctx) -> int:
    b = C.c_size_t()
    load().dgs_workspace_query(ctx, C.byref(b))
    return int(b.value)


def dgs_workspace_query_batch(ctx, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env,
                              max_cams, view_pixel_offset, stream) -> tuple:
    """Direct call of dgs_workspace_query_batch; returns (status, bytes)."""
    b = C.c_size_t()
    rc = load().dgs_workspace_query_batch(ctx, nodes, int(n_nodes), _ptr(env_node_ids), int(n_envs), int(max_nodes),
                                          _ptr(node_poses), cams, _ptr(cams_per_env), int(max_cams),
                                          _ptr(view_pixel_offset), C.byref(b), stream)
    return rc, int(b.value)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if isinstance(a, int):
        return a
    return a.data_ptr()          # torch tensor


def dgs_render(ctx, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env, max_cams,
               out_rgb, out_depth, out_alpha, view_pixel_offset, stream) -> int:
    """Direct call of dgs_render.  Host tables are numpy arrays (or ctypes arrays), device
    buffers are torch tensors or integer device addresses, stream an integer cudaStream_t."""
    return load().dgs_render(ctx, nodes, int(n_nodes), _ptr(env_node_ids), int(n_envs), int(max_nodes),
                             _ptr(node_poses), cams, _ptr(cams_per_env), int(max_cams), _ptr(out_rgb),
                             _ptr(out_depth), _ptr(out_alpha), _ptr(view_pixel_offset), stream)


def dgs_render_backward(ctx, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env,
                        max_cams, out_rgb, out_depth, grad_rgb, grad_depth, grads, grad_poses, view_pixel_offset,
                        stream) -> int:
    """Direct call of dgs_render_backward; `grads` is a ctypes array of dgs_node_grads (or None)."""
    return load().dgs_render_backward(ctx, nodes, int(n_nodes), _ptr(env_node_ids), int(n_envs), int(max_nodes),
                                      _ptr(node_poses), cams, _ptr(cams_per_env), int(max_cams), _ptr(out_rgb),
                                      _ptr(out_depth), _ptr(grad_rgb), _ptr(grad_depth), grads, _ptr(grad_poses),
                                      _ptr(view_pixel_offset), stream)


def dgs_last_stats(ctx) -> dict:
    s = dgs_stats()
    load().dgs_last_stats(ctx, C.byref(s))
    return {k: getattr(s, k) for k, _ in dgs_stats._fields_}


def dgs_kernel_times(ctx) -> dict:
    a = (C.c_float * len(KERNEL_CLASSES))()
    load().dgs_kernel_times(ctx, a)
    return dict(zip(KERNEL_CLASSES, [float(x) for x in a]))


def dgs_last_launches(ctx) -> int:
    return int(load().dgs_last_launches(ctx))


def dgs_build_flags() -> int:
    return int(load().dgs_build_flags())


@contextlib.contextmanager
def using(lib: C.CDLL):
    """Routes every wrapper of this module (and so Renderer and DeviceScene) to `lib`, for
    instance load(DEBUG_LIB_PATH), inside the block.  Contexts made inside must be closed
    inside."""
    global _lib
    prev = load()
    with _lock:
        _lib = lib
    try:
        yield lib
    finally:
        with _lock:
            _lib = prev


def dgs_render_noalloc(opt, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env,
                       max_cams, out_rgb, out_depth, out_alpha, view_pixel_offset, stream) -> int:
    """Direct call of dgs_render_noalloc (no device or pinned memory is allocated by the
    library; its workspace is a fixed 64 MiB device array).  Arguments as dgs_render, with a
    dgs_options structure (or None for the defaults) in place of the context."""
    return load().dgs_render_noalloc(C.byref(opt) if opt is not None else None, nodes, int(n_nodes),
                                     _ptr(env_node_ids), int(n_envs), int(max_nodes), _ptr(node_poses), cams,
                                     _ptr(cams_per_env), int(max_cams), _ptr(out_rgb), _ptr(out_depth),
                                     _ptr(out_alpha), _ptr(view_pixel_offset), stream)


def dgs_autotune(ctx, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env, max_cams,
                 out_rgb, out_depth, out_alpha, view_pixel_offset, candidates, reps, stream):
    """Direct call of dgs_autotune.  `candidates` is a sequence of (tile_w, tile_h) or None for
    the library's default list.  Returns (status, dgs_tune_result)."""
    res = dgs_tune_result()
    if candidates is None:
        cand, nc = None, 0
    else:
        flat = np.ascontiguousarray(np.asarray(candidates, np.int32).reshape(-1, 2))
        cand, nc = flat, len(flat)
    rc = load().dgs_autotune(ctx, nodes, int(n_nodes), _ptr(env_node_ids), int(n_envs), int(max_nodes),
                             _ptr(node_poses), cams, _ptr(cams_per_env), int(max_cams), _ptr(out_rgb),
                             _ptr(out_depth), _ptr(out_alpha), _ptr(view_pixel_offset), _ptr(cand), int(nc),
                             int(reps), C.byref(res), stream)
    return rc, res


def dgs_spatial_order(mean) -> np.ndarray:
    """Direct call of dgs_spatial_order on a host [n,3] FP32 array; returns the int64 permutation."""
    m = np.ascontiguousarray(mean, np.float32).reshape(-1, 3)
    perm = np.empty(len(m), np.int64)
    rc = load().dgs_spatial_order(m.ctypes.data if len(m) else None, len(m), perm.ctypes.data if len(m) else None)
    if rc != DGS_OK:
        raise DgsError(rc, "dgs_spatial_order")
    return perm


def dgs_set_augment(ctx, aug, n_views, overlay, n_frames, overlay_w, overlay_h) -> int:
    """Direct call of dgs_set_augment.  `aug` is a numpy record array with dgs_augment's layout
    (scenes.AUGMENT_DTYPE) or a ctypes array of dgs_augment, or None to clear; `overlay` a uint8
    device tensor [n_frames, overlay_h, overlay_w, 3], an integer device address, or None."""
    if isinstance(aug, np.ndarray):
        assert aug.dtype.itemsize == C.sizeof(dgs_augment) and aug.flags.c_contiguous
    return load().dgs_set_augment(ctx, _ptr(aug) if not isinstance(aug, C.Array) else C.addressof(aug),
                                  int(n_views), _ptr(overlay), int(n_frames), int(overlay_w), int(overlay_h))


def dgs_augment_rgb(ctx, rgb, view_size, view_pixel_offset, n_views, stream) -> int:
    """Direct call of dgs_augment_rgb; view_size is a host int32 [n_views, 2] array of (width, height)."""
    vs = np.ascontiguousarray(view_size, np.int32)
    return load().dgs_augment_rgb(ctx, _ptr(rgb), vs.ctypes.data, _ptr(view_pixel_offset), int(n_views), stream)


def dgs_lidar_build(ctx, nodes, n_nodes, stream) -> int:
    """Direct call of dgs_lidar_build (nodes: ctypes array of dgs_node)."""
    return load().dgs_lidar_build(ctx, nodes, int(n_nodes), stream)


def dgs_lidar_trace(ctx, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, sensors, n_sensors, dirs,
                    n_dirs, r_min, r_max, out_d, out_a, stream) -> int:
    """Direct call of dgs_lidar_trace; `sensors` is a ctypes array of dgs_lidar, `dirs` a device
    tensor [n_dirs, 3] (or address), outputs device tensors [n_sensors * n_dirs]."""
    return load().dgs_lidar_trace(ctx, nodes, int(n_nodes), _ptr(env_node_ids), int(n_envs), int(max_nodes),
                                  _ptr(node_poses), sensors, int(n_sensors), _ptr(dirs), int(n_dirs), float(r_min),
                                  float(r_max), _ptr(out_d), _ptr(out_a), stream)


def lidar_sensors(sensor_env, sensor_pose):
    """ctypes array of dgs_lidar from env indices [S] and world_from_sensor poses [S,3,4]."""
    env = np.asarray(sensor_env, np.int32).reshape(-1)
    pose = np.asarray(sensor_pose, np.float32).reshape(len(env), 12)
    arr = (dgs_lidar * max(len(env), 1))()
    for i in range(len(env)):
        arr[i].env = int(env[i])
        arr[i].world_from_sensor[:] = [float(x) for x in pose[i]]
    return arr


def dgs_mesh_to_gaussians(ctx, vertices, n_vertices, faces, n_faces, vertex_colors, flatten, opacity_logit, sh_degree,
                          out_mean, out_log_scale, out_quat, out_opacity_logit, out_sh, stream) -> int:
    """Direct call of dgs_mesh_to_gaussians (device buffers as torch tensors or addresses)."""
    return load().dgs_mesh_to_gaussians(ctx, _ptr(vertices), int(n_vertices), _ptr(faces), int(n_faces),
                                        _ptr(vertex_colors), float(flatten), float(opacity_logit), int(sh_degree),
                                        _ptr(out_mean), _ptr(out_log_scale), _ptr(out_quat), _ptr(out_opacity_logit),
                                        _ptr(out_sh), stream)


def dgs_tsdf_integrate(ctx, tsdf, weight, nx, ny, nz, origin, voxel, trunc, max_weight, min_alpha, cams, n_views,
                       depth, alpha, view_pixel_offset, stream) -> int:
    """Direct call of dgs_tsdf_integrate; `cams` is a ctypes array of dgs_camera, `origin` 3 floats."""
    org = np.ascontiguousarray(np.asarray(origin, np.float32).reshape(3))
    return load().dgs_tsdf_integrate(ctx, _ptr(tsdf), _ptr(weight), int(nx), int(ny), int(nz), org.ctypes.data,
                                     float(voxel), float(trunc), float(max_weight), float(min_alpha), cams, int(n_views),
                                     _ptr(depth), _ptr(alpha), _ptr(view_pixel_offset), stream)


def cameras(views) -> "C.Array":
    """ctypes array of dgs_camera from (fx, fy, cx, cy, W, H, cam_from_world [3,4]) tuples."""
    arr = (dgs_camera * max(len(views), 1))()
    for k, (fx, fy, cx, cy, w, h, P) in enumerate(views):
        c = arr[k]
        c.fx, c.fy, c.cx, c.cy, c.width, c.height = float(fx), float(fy), float(cx), float(cy), int(w), int(h)
        c.cam_from_world[:] = [float(x) for x in np.asarray(P, np.float32).reshape(12)]
    return arr


def dgs_pose_twist_grad(poses, grad_poses, n, out_twist, stream) -> int:
    """Direct call of dgs_pose_twist_grad: device poses [n,12], their 3x4 gradients [n,12] and the
    output twists [n,6] (torch tensors or device addresses), stream an integer cudaStream_t."""
    return load().dgs_pose_twist_grad(_ptr(poses), _ptr(grad_poses), int(n), _ptr(out_twist), stream)
