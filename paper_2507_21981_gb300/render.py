"""Torch-facing wrapper of libdgs: device memory and streams come from PyTorch, every render
step runs in the CUDA library (dgs.py marshals the arguments)."""
from __future__ import annotations

import copy
import ctypes as C

import numpy as np
import torch

from . import dgs as D

_TORCH_DTYPES = {"f32": (torch.float32, D.DGS_F32), "bf16": (torch.bfloat16, D.DGS_BF16),
                 "f16": (torch.float16, D.DGS_F16)}


class DeviceScene:
    """A scene's nodes resident on the GPU plus the host tables of one batch of envs x cameras.

    Attribute storage: `dtype` in {"f32", "bf16", "f16"} applies to log-scales, quaternions
    and SH coefficients; means and opacity logits stay FP32.

    spatial_order: store every node's Gaussians in the order dgs_spatial_order gives (Z-order of
    the means), applied once here; `perms[k]` maps stored index -> index in `scene`, and
    `scene` is the permuted scene the device arrays hold (gradients come back in that order).
    """

    def __init__(self, scene, device="cuda", dtype: str = "f32", spatial_order: bool = False):
        tdt, code = _TORCH_DTYPES[dtype]
        self.perms = None
        if spatial_order:
            self.perms = [D.dgs_spatial_order(nd.mean) for nd in scene.nodes]
            scene = copy.copy(scene)
            scene.nodes = [nd.subset(p) for nd, p in zip(scene.nodes, self.perms)]
        self.scene = scene
        self.dtype = dtype
        self.device = torch.device(device)
        self.tensors = []
        self.nodes = (D.dgs_node * len(scene.nodes))()
        for k, nd in enumerate(scene.nodes):
            t = dict(mean=torch.as_tensor(np.ascontiguousarray(nd.mean, np.float32), device=self.device),
                     log_scale=torch.as_tensor(np.ascontiguousarray(nd.log_scale, np.float32)).to(self.device, tdt),
                     quat=torch.as_tensor(np.ascontiguousarray(nd.quat, np.float32)).to(self.device, tdt),
                     opacity_logit=torch.as_tensor(np.ascontiguousarray(nd.opacity_logit, np.float32), device=self.device),
                     sh=torch.as_tensor(np.ascontiguousarray(nd.sh, np.float32)).to(self.device, tdt).contiguous())
            self.tensors.append(t)
            n = self.nodes[k]
            n.mean, n.log_scale, n.quat = t["mean"].data_ptr(), t["log_scale"].data_ptr(), t["quat"].data_ptr()
            n.opacity_logit, n.sh = t["opacity_logit"].data_ptr(), t["sh"].data_ptr()
            n.n, n.sh_degree, n.dtype = nd.n, nd.sh_degree, code
        self.n_nodes = len(scene.nodes)
        self.env_node_ids = np.ascontiguousarray(scene.env_node_ids, np.int32)
        self.n_envs, self.max_nodes = self.env_node_ids.shape
        self.cams_per_env = np.ascontiguousarray(scene.cams_per_env, np.int32)
        self.max_cams = int(scene.cam_res.shape[1])
        E, Cm = self.n_envs, self.max_cams
        self.cams = (D.dgs_camera * (E * Cm))()
        self.view_res = []
        for e in range(E):
            for c in range(Cm):
                cam = self.cams[e * Cm + c]
                fx, fy, cx, cy = (float(x) for x in scene.cam_intr[e, c])
                cam.fx, cam.fy, cam.cx, cam.cy = fx, fy, cx, cy
                w, h = (int(x) for x in scene.cam_res[e, c])
                cam.width, cam.height = max(w, 1), max(h, 1)
                cam.cam_from_world[:] = [float(x) for x in np.asarray(scene.cam_pose[e, c], np.float64).reshape(12)]
                if c < self.cams_per_env[e]:
                    self.view_res.append((w, h))
        self.n_views = len(self.view_res)
        self.n_pixels = int(sum(w * h for w, h in self.view_res))
        self.view_offsets = np.concatenate([[0], np.cumsum([w * h for w, h in self.view_res])]).astype(np.int64)
        self.node_poses = torch.as_tensor(np.ascontiguousarray(scene.node_poses, np.float32).reshape(E, self.max_nodes, 12),
                                          device=self.device)

    PARAM_NAMES = ("mean", "log_scale", "quat", "opacity_logit", "sh")

    def param_list(self):
        """The attribute tensors, node by node, in PARAM_NAMES order."""
        return [t[name] for t in self.tensors for name in self.PARAM_NAMES]

    def set_poses(self, node_poses):
        """Copy new per-env node poses ([E,K,3,4] or [E,K,12]) into the scene's pose buffer (in
        place, so a captured render graph keeps reading the same device array)."""
        src = torch.as_tensor(node_poses, dtype=torch.float32).reshape(self.n_envs, self.max_nodes, 12)
        if src.data_ptr() != self.node_poses.data_ptr():
            self.node_poses.copy_(src, non_blocking=False)

    def view_slice(self, v: int):
        return slice(int(self.view_offsets[v]), int(self.view_offsets[v + 1]))


_MODES = {"plain": D.DGS_MODE_PLAIN, "batched": D.DGS_MODE_BATCHED, "graph": D.DGS_MODE_GRAPH}


class Renderer:
    """A libdgs context.  Options are the fields of dgs_options (see include/dgs.h).

    mode "graph" replays a captured CUDA graph of the whole render when the batch keeps its
    structure and buffers; render() then returns output tensors owned by the Renderer (the
    same storage every call, overwritten by the next render) unless `out` is given."""

    def __init__(self, mode: str = "batched", tile=(16, 16), profile: int = 0, **opts):
        o = D.dgs_default_options()
        o.mode = _MODES[mode]
        self.mode = mode
        self._outs = None
        o.tile_w, o.tile_h = int(tile[0]), int(tile[1])
        o.profile = int(profile)
        for k, v in opts.items():
            if k == "bg":
                o.bg = (C.c_float * 3)(*[float(x) for x in v])
            else:
                setattr(o, k, v)
        self.options = o
        self._aug = None
        self._lib = D.load()            # the library the context belongs to (see dgs.using)
        self.tune_cached = False        # the last autotune took its shape from a TuneCache
        self.ctx = D.dgs_context_create(o)

    def set_options(self, **opts):
        """Changes fields of the context's dgs_options (dgs_set_options); raises if invalid."""
        o = D.dgs_options.from_buffer_copy(self.options)
        for k, v in opts.items():
            if k == "bg":
                o.bg = (C.c_float * 3)(*[float(x) for x in v])
            else:
                setattr(o, k, v)
        rc = D.dgs_set_options(self.ctx, o)
        if rc != D.DGS_OK:
            raise D.DgsError(rc, D.dgs_last_error(self.ctx))
        self.options = o

    def close(self):
        if self.ctx:
            self._lib.dgs_context_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, ds: DeviceScene, out=None, with_alpha: bool = True, stream=None):
        """Renders every view of `ds`; returns (rgb [P,3], depth [P], alpha [P] or None), flat over views."""
        rgb, depth, alpha = out if out is not None else self._outputs(ds, with_alpha)
        s = stream if stream is not None else torch.cuda.current_stream(ds.device)
        rc = D.dgs_render(self.ctx, ds.nodes, ds.n_nodes, ds.env_node_ids, ds.n_envs, ds.max_nodes, ds.node_poses,
                          ds.cams, ds.cams_per_env, ds.max_cams, rgb, depth, alpha, None, s.cuda_stream)
        if rc != D.DGS_OK:
            raise D.DgsError(rc, D.dgs_last_error(self.ctx))
        return rgb, depth, alpha

    def set_augment(self, params=None, overlay=None):
        """Sets the per-view image randomisation that every later render applies to its RGB
        (dgs_set_augment): `params` a record array with dgs_augment's fields (one per view), or
        None to clear; `overlay` a uint8 CUDA tensor [frames, height, width, 3] (kept alive
        here while the randomisation is set)."""
        if params is None:
            rc = D.dgs_set_augment(self.ctx, None, 0, None, 0, 0, 0)
            self._aug = None
        else:
            prm = np.ascontiguousarray(params)
            if overlay is not None:
                assert overlay.dtype == torch.uint8 and overlay.is_cuda and overlay.dim() == 4 and overlay.shape[3] == 3
                overlay = overlay.contiguous()
                nf, oh, ow = (int(x) for x in overlay.shape[:3])
            else:
                nf = oh = ow = 0
            rc = D.dgs_set_augment(self.ctx, prm, len(prm), overlay, nf, ow, oh)
            if rc == D.DGS_OK:
                self._aug = (prm, overlay)
        if rc != D.DGS_OK:
            raise D.DgsError(rc, D.dgs_last_error(self.ctx))

    def augment_rgb(self, ds: DeviceScene, rgb, stream=None):
        """Applies the randomisation set by set_augment to `rgb` ([P,3] FP32 CUDA, flat over the
        views of `ds`) in place, as a separate kernel (dgs_augment_rgb)."""
        s = stream if stream is not None else torch.cuda.current_stream(ds.device)
        sizes = np.asarray(ds.view_res, np.int32).reshape(-1, 2)
        rc = D.dgs_augment_rgb(self.ctx, rgb, sizes, None, ds.n_views, s.cuda_stream)
        if rc != D.DGS_OK:
            raise D.DgsError(rc, D.dgs_last_error(self.ctx))
        return rgb

    def lidar_build(self, ds: DeviceScene, stream=None):
        """Builds the LiDAR ray-tracing structures of the scene's nodes (dgs_lidar_build)."""
        s = stream if stream is not None else torch.cuda.current_stream(ds.device)
        rc = D.dgs_lidar_build(self.ctx, ds.nodes, ds.n_nodes, s.cuda_stream)
        if rc != D.DGS_OK:
            raise D.DgsError(rc, D.dgs_last_error(self.ctx))

    def lidar_trace(self, ds: DeviceScene, sensor_env, sensor_pose, dirs, r_min: float = 0.05, r_max: float = 30.0,
                    out=None, stream=None):
        """Traces every (sensor, direction) ray (dgs_lidar_trace): sensor_env [S], sensor_pose
        [S,3,4] world_from_sensor, dirs a CUDA tensor [J,3] of sensor-frame directions.  Returns
        (D, A) CUDA tensors [S, J]: D = sum w t* (range = D / A), A = 1 - T."""
        sensors = sensor_env if isinstance(sensor_env, C.Array) else D.lidar_sensors(sensor_env, sensor_pose)
        S = len(sensors) if isinstance(sensor_env, C.Array) else len(np.asarray(sensor_env).reshape(-1))
        J = int(dirs.shape[0])
        if out is None:
            out = (torch.empty((S, J), dtype=torch.float32, device=ds.device),
                   torch.empty((S, J), dtype=torch.float32, device=ds.device))
        s = stream if stream is not None else torch.cuda.current_stream(ds.device)
        rc = D.dgs_lidar_trace(self.ctx, ds.nodes, ds.n_nodes, ds.env_node_ids, ds.n_envs, ds.max_nodes,
                               ds.node_poses, sensors, S, dirs, J, r_min, r_max, out[0], out[1], s.cuda_stream)
        if rc != D.DGS_OK:
            raise D.DgsError(rc, D.dgs_last_error(self.ctx))
        return out

    def mesh_to_gaussians(self, vertices, faces, vertex_colors=None, flatten: float = 0.01,
                          opacity_logit: float = 2.0, sh_degree: int = 0, stream=None) -> dict:
        """One flat Gaussian per facet (dgs_mesh_to_gaussians): vertices [V,3] FP32 and faces
        [F,3] int32 CUDA tensors (colours [V,3] or None).  Returns CUDA tensors in the node
        layout: mean, log_scale, quat, opacity_logit, sh [F, (deg+1)^2, 3]."""
        F = int(faces.shape[0])
        dev = vertices.device
        nc = (sh_degree + 1) ** 2
        out = dict(mean=torch.empty((F, 3), device=dev), log_scale=torch.empty((F, 3), device=dev),
                   quat=torch.empty((F, 4), device=dev), opacity_logit=torch.empty((F,), device=dev),
                   sh=torch.empty((F, nc, 3), device=dev))
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        rc = D.dgs_mesh_to_gaussians(self.ctx, vertices, int(vertices.shape[0]), faces, F, vertex_colors, flatten,
                                     opacity_logit, sh_degree, out["mean"], out["log_scale"], out["quat"],
                                     out["opacity_logit"], out["sh"], s.cuda_stream)
        if rc != D.DGS_OK:
            raise D.DgsError(rc, D.dgs_last_error(self.ctx))
        return out

    def _outputs(self, ds: DeviceScene, with_alpha: bool):
        def fresh():
            return (torch.empty((ds.n_pixels, 3), dtype=torch.float32, device=ds.device),
                    torch.empty((ds.n_pixels,), dtype=torch.float32, device=ds.device),
                    torch.empty((ds.n_pixels,), dtype=torch.float32, device=ds.device) if with_alpha else None)
        if self.mode != "graph":
            return fresh()
        o = self._outs
        if o is None or o[1].numel() != ds.n_pixels or o[1].device != ds.device or (o[2] is not None) != with_alpha:
            self._outs = o = fresh()
        return o

    def autotune(self, ds: DeviceScene, candidates=None, reps: int = 3, out=None, with_alpha: bool = True,
                 stream=None, cache: "TuneCache | None" = None):
        """Times dgs_render of `ds` with each candidate tile shape ((w, h) pairs; None = the
        library's list), keeps the fastest on this context and renders once with it.
        Returns (best (w, h), {(w, h): ms per render}, (rgb, depth, alpha)).  With `cache`, a
        batch whose class (GPU, resolutions, Gaussian density) the cache holds takes the cached
        shape and renders once without timing; a new class is timed and stored.
        self.tune_cached tells which happened."""
        rgb, depth, alpha = out if out is not None else self._outputs(ds, with_alpha)
        s = stream if stream is not None else torch.cuda.current_stream(ds.device)
        self.tune_cached = False
        if cache is not None:
            key = TuneCache.key(ds, torch.cuda.get_device_name(ds.device))
            hit = cache.get(key)
            if hit is not None:
                best, times = hit
                self.set_options(tile_w=best[0], tile_h=best[1])
                self.tune_cached = True
                return best, times, self.render(ds, out=(rgb, depth, alpha), stream=s)
        rc, res = D.dgs_autotune(self.ctx, ds.nodes, ds.n_nodes, ds.env_node_ids, ds.n_envs, ds.max_nodes,
                                 ds.node_poses, ds.cams, ds.cams_per_env, ds.max_cams, rgb, depth, alpha, None,
                                 candidates, reps, s.cuda_stream)
        if rc != D.DGS_OK:
            raise D.DgsError(rc, D.dgs_last_error(self.ctx))
        times = {(res.tile_w[i], res.tile_h[i]): float(res.ms[i]) for i in range(res.n)}
        best = (res.tile_w[res.best], res.tile_h[res.best])
        self.options.tile_w, self.options.tile_h = best
        if cache is not None:
            cache.put(key, best, times)
        return best, times, (rgb, depth, alpha)

    def backward(self, ds: DeviceScene, out_rgb, out_depth, grad_rgb, grad_depth=None, want_poses: bool = True,
                 stream=None, out: "GradBuffers | None" = None):
        """Gradients of L = sum(grad_rgb * rgb) + sum(grad_depth * depth) for the render of `ds`.

        Returns (list of per-node dicts of FP32 tensors mean/log_scale/quat/opacity_logit/sh,
        pose gradient [E,K,3,4] or None).  With `out` (GradBuffers(ds) made once) the
        gradients are written into its buffers, zeroed first, and those are returned: the next
        backward with the same `out` overwrites them."""
        gb = GradBuffers(ds, want_poses) if out is None else out
        if out is not None:
            gb.flat.zero_()
        s = stream if stream is not None else torch.cuda.current_stream(ds.device)
        grad_rgb = grad_rgb.contiguous().float()
        grad_depth = None if grad_depth is None else grad_depth.contiguous().float()
        rc = D.dgs_render_backward(self.ctx, ds.nodes, ds.n_nodes, ds.env_node_ids, ds.n_envs, ds.max_nodes,
                                   ds.node_poses, ds.cams, ds.cams_per_env, ds.max_cams, out_rgb, out_depth, grad_rgb,
                                   grad_depth, gb.arr, gb.gposes, None, s.cuda_stream)
        if rc != D.DGS_OK:
            raise D.DgsError(rc, D.dgs_last_error(self.ctx))
        return gb.node_grads, (None if gb.gposes is None else gb.gposes.view(ds.n_envs, ds.max_nodes, 3, 4))

    def stats(self) -> dict:
        return D.dgs_last_stats(self.ctx)

    def kernel_times(self) -> dict:
        return D.dgs_kernel_times(self.ctx)

    def launches(self) -> int:
        return D.dgs_last_launches(self.ctx)

    def workspace_bytes(self) -> int:
        return D.dgs_workspace_query(self.ctx)


class TuneCache:
    """Tile shapes found by Renderer.autotune, kept in a JSON file keyed by (GPU name,
    resolution class, Gaussian density).  The resolution class is the sorted set of the batch's
    view resolutions and its view count rounded to a power of two; the density is the Gaussians
    present per view, rounded to a power of two.  A batch of a known class then starts with its
    tile shape without timing the candidates again.  The file is rewritten whole (through a
    temporary file and a rename) on every store."""

    def __init__(self, path: str):
        self.path = path

    @staticmethod
    def key(ds: DeviceScene, device_name: str) -> str:
        def p2(x: float) -> int:
            return 1 << max(0, int(round(np.log2(max(x, 1.0)))))
        res = ",".join(f"{w}x{h}" for w, h in sorted(set(ds.view_res)))
        per_view = ds.scene.instances() / max(ds.n_views, 1)
        return f"{device_name}|res={res}|views~{p2(ds.n_views)}|gaussians_per_view~{p2(per_view)}"

    def _load(self) -> dict:
        import json
        import os
        if not os.path.exists(self.path):
            return {}
        with open(self.path) as f:
            return json.load(f)

    def get(self, key: str):
        """(best (w, h), {(w, h): ms}) stored for `key`, or None."""
        e = self._load().get(key)
        if e is None:
            return None
        times = {tuple(int(v) for v in k.split("x")): float(ms) for k, ms in e["ms"].items()}
        return (int(e["best"][0]), int(e["best"][1])), times

    def put(self, key: str, best, times) -> None:
        import json
        import os
        data = self._load()
        data[key] = {"best": [int(best[0]), int(best[1])],
                     "ms": {f"{int(w)}x{int(h)}": float(ms) for (w, h), ms in times.items()}}
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


class GradBuffers:
    """Gradient outputs of Renderer.backward for one DeviceScene: one zero-filled FP32 buffer
    holding every node's attribute gradients (and the pose gradient), its per-node views and
    the dgs_node_grads table of their addresses.  Made once and passed as `out`, it spares each
    backward the allocation and the view set-up."""

    NAMES = ("mean", "log_scale", "quat", "opacity_logit", "sh")

    def __init__(self, ds: DeviceScene, want_poses: bool = True):
        sizes = [t[name].numel() for t in ds.tensors for name in self.NAMES]
        n_pose = ds.n_envs * ds.max_nodes * 12 if want_poses else 0
        self.flat = torch.zeros(sum(sizes) + n_pose, dtype=torch.float32, device=ds.device)
        self.arr = (D.dgs_node_grads * ds.n_nodes)()
        self.node_grads = []
        parts = torch.split(self.flat, sizes + ([n_pose] if n_pose else []))
        base = self.flat.data_ptr()
        off = 0
        for k, t in enumerate(ds.tensors):
            g = {}
            for j, name in enumerate(self.NAMES):
                g[name] = parts[5 * k + j].view(t[name].shape)
                setattr(self.arr[k], name, base + 4 * off)
                off += sizes[5 * k + j]
            self.node_grads.append(g)
        self.gposes = parts[-1].view(ds.n_envs, ds.max_nodes, 12) if n_pose else None


class DGSRenderFn(torch.autograd.Function):
    """Differentiable render of a DeviceScene.

    apply(renderer, ds, node_poses, *params) -> (rgb [P,3], depth [P], alpha [P]), where params
    are the scene's own attribute tensors in DeviceScene.param_list() order (the C ABI reads them
    in place) and node_poses is [E,K,3,4] or [E,K,12] FP32 on the device.  Gradients flow to
    every param and to node_poses through dgs_render_backward; alpha carries no gradient.
    """

    @staticmethod
    def forward(ctx, renderer, ds, node_poses, *params):
        ds.set_poses(node_poses.detach())
        rgb, depth, alpha = renderer.render(ds)
        ctx.renderer, ctx.ds = renderer, ds
        ctx.save_for_backward(rgb, depth)
        ctx.pose_shape = node_poses.shape
        ctx.mark_non_differentiable(alpha)
        return rgb, depth, alpha

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_alpha):
        rgb, depth = ctx.saved_tensors
        ds = ctx.ds
        if g_rgb is None:
            g_rgb = torch.zeros_like(rgb)
        node_grads, gposes = ctx.renderer.backward(ds, rgb, depth, g_rgb, g_depth)
        flat = []
        for k, t in enumerate(ds.tensors):
            for name in DeviceScene.PARAM_NAMES:
                flat.append(node_grads[k][name].to(t[name].dtype))
        return (None, None, gposes.reshape(ctx.pose_shape)) + tuple(flat)


def render_differentiable(renderer: Renderer, ds: DeviceScene, node_poses=None):
    """Convenience wrapper: renders with gradients to the scene tensors (which should have
    requires_grad set) and to node_poses (defaults to the scene's current poses)."""
    poses = ds.node_poses if node_poses is None else node_poses
    return DGSRenderFn.apply(renderer, ds, poses, *ds.param_list())


def pose_twist_grad(node_poses: torch.Tensor, grad_poses: torch.Tensor) -> torch.Tensor:
    """se(3) gradient (rho, phi) of a left perturbation of each pose, from the 3x4 pose gradient
    (dgs_pose_twist_grad on the current stream).  node_poses, grad_poses: CUDA FP32 [..., 3, 4]
    (or [..., 12]); returns [..., 6]."""
    p = node_poses.detach().reshape(-1, 12).to(torch.float32).contiguous()
    g = grad_poses.detach().reshape(-1, 12).to(torch.float32).contiguous()
    if p.shape != g.shape or not p.is_cuda or not g.is_cuda:
        raise ValueError("pose_twist_grad: poses and gradients must be CUDA tensors of the same shape")
    out = torch.empty((p.shape[0], 6), device=p.device, dtype=torch.float32)
    rc = D.dgs_pose_twist_grad(p, g, p.shape[0], out, torch.cuda.current_stream(p.device).cuda_stream)
    if rc != D.DGS_OK:
        raise D.DgsError(rc, "dgs_pose_twist_grad")
    return out.reshape(*node_poses.shape[:-2] if node_poses.shape[-2:] == (3, 4) else node_poses.shape[:-1], 6)
