"""Benchmark: batched 3DGS RGB+depth rendering of many environments on one GB300 per rank.

Workload (one step = one dgs_render call over every view of the batch): 64 envs x 2 cameras
at 640x480, a shared 1M-Gaussian SH-3 room (background node) plus 4 object nodes x 20k
Gaussians at per-env SE(3) poses, FP32 attributes.  Synthetic, seeded scenes stand in for the
paper's scanned rooms and objects.  Under torchrun every rank renders its own batch (weak
scaling, no collective on the data path) and rank 0 reports the sum over ranks.

Prints one JSON line.  `value` is batched Mpix/s with inputs resident in HBM; `e2e` is the
same metric through the C ABI with host buffers (poses uploaded from pinned memory, RGB+depth
read back to pinned memory inside the timed region).  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpix/s RGB+depth batched vs plain per-view; fwd+bwd ms/view at 500k Gaussians"
# FP32 operations of one (pixel, Gaussian) evaluation inside the ellipse: offsets 2, factored
# quadratic form 5, compare 1, exp argument + MUFU 2, opacity product + clamp 2, alpha test 1,
# transmittance 2, termination test 1, weight 1, colour 3, depth 1 (about 20).
OPS_PER_PAIR = 21
# The adjoint of one composited (pixel, Gaussian) pair: the forward's evaluation replayed (21),
# prefix sums (4), reciprocal and normalised remainders (5), dL/dalpha (8), colour and depth
# partials (4), opacity and quadratic-form partials (8): about 50.
BWD_OPS_PER_PAIR = 50
# Projection of one visible instance: faithfully rounded camera-space centre (3 compensated dot
# products, 105), guarded Jacobian and 2D covariance by Cauchy-Binet (75), conic, centre and
# pixel box (20); spherical-harmonics colour of degree 3: basis (30), 48 FMA, direction (10).
# The count pass runs the conservative per-Gaussian cull and box bound (35: three FMA chains and
# their error bounds, a reciprocal, two square roots, the box and its tiles) instead of the exact
# projection.  The count and emit rates count only per-emitted-instance work: the chunk culls,
# the culled instances' tests and the tile-row runs of emission are left out, so their
# fractions are lower bounds.
PROJ_OPS, SH3_OPS, CULL_OPS = 200, 90, 35
# The projection adjoint moves per visible instance: 40 B of partials, 236 B of FP32 attributes
# read, 236 B of attribute gradients accumulated and 8 B of identity.
PROJECT_BWD_BYTES = 40 + 236 + 236 + 8
# DRAM bytes (read + write) per launch on the full workload, from a one-pass ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the full launch: 1005.0 + 754.6 MB.  Set to
# None whenever the kernel changes after its capture.
TRAFFIC = {"composite": 1.7596e9}
# FP32 operations per (voxel, view) of the TSDF fusion: camera-space point (9 FMA), reciprocal,
# projection (4), bounds (4 compares), coverage test, normalised depth (2), sdf, truncation,
# clamp (2), running average (3), weight update (2)
TSDF_OPS = 30
WORKLOAD = "64 envs x 2 cams 640x480, 1M-Gaussian SH3 room + 4 objects x 20k at per-env poses (config 2)"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_scene(rank: int, envs: int, **kw):
    """Weak scaling: rank r renders its own batch of `envs` environments of the benchmark law
    (seed 1 + r); no data crosses ranks."""
    from paper_2507_21981_gb300 import scenes
    return scenes.config2(seed=1 + rank, n_envs=envs, **kw)


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The slowest rank's time (the only collective of the benchmark)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every `period_ms` in the background.

    Start it before the warm-up (nvidia-smi needs a moment to start) and bracket each timed
    region with mark_start() / mark_end(): the summary keeps the samples whose own nvidia-smi
    timestamps fall inside those windows.  If none can be placed (a timestamp that does not
    parse), it keeps every sample taken while the sampler ran and says so in `window`."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.gpu = gpu_index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []
        self.windows = []
        self._t0 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark_start(self):
        self._t0 = time.time()

    def mark_end(self):
        if self._t0 is not None:
            self.windows.append((self._t0, time.time()))
            self._t0 = None

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.reader.join(timeout=5)

    @staticmethod
    def _when(stamp: str):
        import datetime
        try:
            return datetime.datetime.strptime(stamp.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self):
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                sm, mx = float(f[2]), float(f[3])
            except ValueError:
                continue
            rows.append((self._when(f[0]), sm, mx, {n for n, v in zip(self.REASONS, f[6:10]) if v.lower() == "active"}))
        inside = [r for r in rows if r[0] is not None and any(a <= r[0] <= b for a, b in self.windows)]
        window = "timed region"
        if not inside:
            inside, window = rows, "whole sampling (no sample placed in the timed region)"
        sm = [r[1] for r in inside]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": inside[-1][2] if inside else None,
                "reasons": sorted(set().union(*(r[3] for r in inside))), "samples": len(sm), "window": window}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fwd_bwd_500k(dev, warmup, steps):
    """Forward + backward of one 800x800 view of 500k SH-3 Gaussians (300k room + 8 x 25k posed
    objects): render, then dL/d(all attributes, poses) for a fixed upstream gradient, as a
    training step runs it: the forward a graph replay, the backward differentiating the tile
    lists its forward kept (keep_lists) into gradient buffers made once.  Beside it, the same
    step with an eager forward, and with the default backward that bins the batch again into
    fresh buffers.  The timed steps run without per-kernel events; kernel times per class come
    from a separate profiled run, and one instrumented forward and backward count the reached
    pairs and the adjoint's atomics."""
    import torch
    from paper_2507_21981_gb300 import scenes
    from paper_2507_21981_gb300.render import DeviceScene, GradBuffers, Renderer
    sc = scenes.config4(seed=1)
    ds = DeviceScene(sc, device=dev, spatial_order=True)
    gen = torch.Generator(device=dev).manual_seed(0)
    g_rgb = torch.randn((ds.n_pixels, 3), device=dev, generator=gen)
    g_d = torch.randn((ds.n_pixels,), device=dev, generator=gen)
    stream = torch.cuda.current_stream(dev)
    gb = GradBuffers(ds)

    def timed(r, out, n):
        def step():
            rgb, depth, _ = r.render(ds)
            r.backward(ds, rgb, depth, g_rgb, g_d, out=out)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        path = r.stats()["path"]
        r.close()
        return e0.elapsed_time(e1) / n, path
    ms, path = timed(Renderer(mode="graph", keep_lists=1), gb, steps)
    assert path == 4, "the backward did not use the kept lists"
    ms_eager, _ = timed(Renderer(mode="batched", keep_lists=1), gb, steps)
    ms_rebuild, _ = timed(Renderer(mode="batched"), None, steps)
    # kernel times per class (library events) of the eager kept-lists step
    r = Renderer(mode="batched", profile=True, keep_lists=1)
    kt = {}
    for i in range(warmup + steps):
        rgb, depth, _ = r.render(ds)
        fk = r.kernel_times()
        r.backward(ds, rgb, depth, g_rgb, g_d, out=gb)
        bk = r.kernel_times()
        if i >= warmup:
            for k, v in fk.items():
                kt["fwd_" + k] = kt.get("fwd_" + k, 0.0) + v
            for k, v in bk.items():
                kt["bwd_" + k] = kt.get("bwd_" + k, 0.0) + v
    r.close()
    ri = Renderer(mode="batched", profile=2, keep_lists=1)
    rgb, depth, _ = ri.render(ds)
    fwd = ri.stats()
    ri.backward(ds, rgb, depth, g_rgb, g_d)
    bwd = ri.stats()
    ri.close()
    return {"ms": ms, "ms_eager_forward": ms_eager, "ms_lists_binned_again": ms_rebuild, "views": 1,
            "gaussians": sc.n_gaussians, "resolution": "800x800", "steps": steps,
            "kernel_ms": {k: v / steps for k, v in kt.items() if v > 0},
            "work": {"visible": fwd["n_visible"], "pairs": fwd["n_pairs"], "pairs_reached": fwd["px_reached"],
                     "pairs_composited": fwd["px_composited"], "bwd_reductions": bwd["bwd_reductions"]}}


def _time_renders(r, ds, out, steps, stream):
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        r.render(ds, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps


def ragged_graph(dev, warmup, steps):
    """The uneven batch (256 envs, 1-12 of 64 assets of 5k-200k Gaussians each, 1-3 cameras at
    320x240 / 640x480 / 1280x720, 500k-Gaussian room): tile shape picked by dgs_autotune, then
    timed as graph replays."""
    import torch
    from paper_2507_21981_gb300 import scenes
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = scenes.config3(seed=1)
    ds = DeviceScene(sc, device=dev, spatial_order=True)
    out = (torch.empty((ds.n_pixels, 3), device=dev), torch.empty((ds.n_pixels,), device=dev), None)
    r = Renderer(mode="graph")
    best, times, _ = r.autotune(ds, reps=2, out=out)
    for _ in range(warmup):
        r.render(ds, out=out)
    ms = _time_renders(r, ds, out, steps, torch.cuda.current_stream(dev))
    st = r.stats()
    re = Renderer(mode="batched", tile=best)         # the eager sequence (two pipelined view groups)
    for _ in range(warmup):
        re.render(ds, out=out)
    ms_eager = _time_renders(re, ds, out, steps, torch.cuda.current_stream(dev))
    groups = re.stats()["n_groups"]
    re.close()
    res = {"workload": "256 envs, 1-12 assets (5k-200k) + 500k room, 1-3 cams of 320x240/640x480/1280x720 (config 3)",
           "views": ds.n_views, "pixels_per_step": ds.n_pixels, "gaussians": sc.n_gaussians,
           "instances": st["n_instances"], "pairs": st["n_pairs"], "mode": "graph",
           "path": {0: "eager", 1: "graph", 2: "captured", 3: "regrown"}[st["path"]],
           "tile": f"{best[0]}x{best[1]}", "autotune_ms": {f"{w}x{h}": t for (w, h), t in times.items()},
           "ms_per_step": ms, "mpix_s": ds.n_pixels / (ms / 1e3) / 1e6, "steps": steps,
           "eager_mpix_s": ds.n_pixels / (ms_eager / 1e3) / 1e6, "eager_groups": groups}
    r.close()
    return res


def precision_scale(dev, warmup, steps):
    """3M-Gaussian room + 6 objects x 50k, 128 envs x 3 cameras 640x480, with log-scales,
    quaternions and SH stored in FP32, BF16 and FP16 (means, opacities and all arithmetic FP32)."""
    import torch
    from paper_2507_21981_gb300 import scenes
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = scenes.config5(seed=1)
    res = {"workload": "128 envs x 3 cams 640x480, 3M-Gaussian SH3 room + 6 objects x 50k (config 5)",
           "views": sc.n_views, "pixels_per_step": sc.n_pixels, "gaussians": sc.n_gaussians, "steps": steps}
    for dt in ("bf16", "f16", "f32"):
        ds = DeviceScene(sc, device=dev, dtype=dt, spatial_order=True)
        out = (torch.empty((ds.n_pixels, 3), device=dev), torch.empty((ds.n_pixels,), device=dev), None)
        r = Renderer(mode="graph")
        for _ in range(warmup):
            r.render(ds, out=out)
        ms = _time_renders(r, ds, out, steps, torch.cuda.current_stream(dev))
        res[dt] = {"ms_per_step": ms, "mpix_s": ds.n_pixels / (ms / 1e3) / 1e6,
                   "attribute_bytes": int(sum(t.numel() * t.element_size() for d in ds.tensors for t in d.values()))}
        res["pairs"] = r.stats()["n_pairs"]
        r.close()
        del ds, out
        torch.cuda.empty_cache()
    return res


def augment_leg(dev, ds, tile, out, warmup, steps, ms_plain_render):
    """Image randomisation on the benchmark batch (overlay crops of a seeded 8-frame 1280x720
    clip blended into half of the views, HSV jitter and gamma on all): the render with the
    randomisation fused into the compositor, and the separate in-place pass over the same
    RGB (HBM-bound: 24 B of RGB per pixel plus 3 B of overlay where the weight is non-zero)."""
    import numpy as np
    import torch
    from paper_2507_21981_gb300 import dgs as D
    from paper_2507_21981_gb300 import scenes
    from paper_2507_21981_gb300.render import Renderer
    n_f, ow, oh = 8, 1280, 720
    ov = torch.as_tensor(scenes.overlay_frames(1, n_frames=n_f, width=ow, height=oh)).to(dev)
    prm = scenes.augment_params(1, ds.n_views, n_f, ow, oh)
    stream = torch.cuda.current_stream(dev)
    r = Renderer(mode="batched", tile=tile)
    r.set_augment(prm, ov)
    for _ in range(warmup):
        r.render(ds, out=out)
    ms_fused = _time_renders(r, ds, out, steps, stream)
    sizes = np.asarray(ds.view_res, np.int32)
    rgb = out[0]
    for _ in range(warmup):
        r.augment_rgb(ds, rgb)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(steps):
        rc = D.dgs_augment_rgb(r.ctx, rgb, sizes, None, ds.n_views, stream.cuda_stream)
        assert rc == D.DGS_OK
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms_sep = ev0.elapsed_time(ev1) / steps
    r.close()
    px = np.asarray([w * h for w, h in ds.view_res], np.int64)
    px_ov = int(px[prm["overlay_beta"] > 0].sum())
    sep_bytes = ds.n_pixels * 24 + px_ov * 3
    peaks, kind = _peaks()
    gbs = sep_bytes / (ms_sep / 1e3) / 1e9
    # the oracle's randomisation of one view (numpy FP64, one host thread)
    import oracle
    x = np.random.default_rng(0).uniform(0, 1, size=(480, 640, 3))
    ovh = ov[:1].cpu().numpy()
    q = dict(zip(oracle.augment.FIELDS, [prm[0][f] for f in oracle.augment.FIELDS]))
    q["overlay_beta"], q["overlay_frame"] = 0.3, 0
    t0 = time.perf_counter()
    oracle.augment.augment_view(x, q, ovh)
    t_or = time.perf_counter() - t0
    return {"workload": "benchmark batch + per-view randomisation, overlay clip 8 x 1280x720 uint8, "
                        f"{int((prm['overlay_beta'] > 0).sum())} of {ds.n_views} views blended",
            "fused_ms_per_step": ms_fused, "fused_mpix_s": ds.n_pixels / (ms_fused / 1e3) / 1e6,
            "render_ms_per_step_without": ms_plain_render,
            "fused_overhead_pct": 100.0 * (ms_fused - ms_plain_render) / ms_plain_render,
            "separate_pass": {"ms": ms_sep, "bytes": sep_bytes, "gb_s": gbs, "peak_gb_s": peaks["hbm_gbs"],
                              "frac": gbs / peaks["hbm_gbs"], "peak_source": f"{kind} MEASURED_PEAKS.json hbm_gbs",
                              "bytes_per_pixel": "24 (+3 with overlay)"},
            "oracle_mpix_s": 640 * 480 / t_or / 1e6, "oracle_sample": "one 640x480 view, numpy FP64, 1 thread",
            "steps": steps}


def lidar_leg(dev, ds, warmup, steps):
    """LiDAR by Gaussian ray tracing on the benchmark scene: one 32-beam spinning sensor per env
    (32 x 1024 rays over 360 degrees, -30.7 to +10.7 degrees elevation, 0.05-30 m), mounted near
    the workspace; one dgs_lidar_trace call traces all 64 sensors (2.1M rays)."""
    import numpy as np
    import torch
    from paper_2507_21981_gb300 import scenes
    from paper_2507_21981_gb300.render import Renderer
    se, sp = scenes.lidar_sensors(1, ds.n_envs)
    dirs_h = scenes.lidar_pattern(32, 1024)
    dirs = torch.as_tensor(dirs_h).to(dev)
    r = Renderer()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    r.lidar_build(ds)
    build_ms = (time.perf_counter() - t0) * 1e3
    out = (torch.empty((len(se), len(dirs_h)), device=dev), torch.empty((len(se), len(dirs_h)), device=dev))
    for _ in range(warmup):
        r.lidar_trace(ds, se, sp, dirs, out=out)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(steps):
        r.lidar_trace(ds, se, sp, dirs, out=out)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / steps
    a = out[1]
    rays = len(se) * len(dirs_h)
    rp = Renderer(profile=1)
    rp.lidar_build(ds)
    rp.lidar_trace(ds, se, sp, dirs, out=out)
    k_ms = rp.kernel_times()["lidar"]
    rp.close()
    res = {"workload": f"{len(se)} sensors x 32 x 1024 rays (one per env), benchmark scene (1.08M Gaussians per env)",
           "rays_per_step": rays, "ms_per_step": ms, "kernel_ms": k_ms, "mrays_s": rays / ms / 1e3,
           "sensor_frames_s": len(se) * 1e3 / ms, "build_ms": build_ms,
           "returns_frac": float((a > 0.5).float().mean()), "steps": steps}
    r.close()
    # the oracle on a sample of one sensor's rays (host cores)
    import oracle
    from oracle import lidar as OL
    js = np.random.default_rng(0).choice(len(dirs_h), 256, replace=False)
    pk = oracle.oracle._Packed(ds.scene)
    t0 = time.perf_counter()
    OL.trace(ds.scene, se[:1], sp[:1], dirs_h[js], packed=pk)
    dt = time.perf_counter() - t0
    res["oracle_mrays_s"] = 256 / dt / 1e6
    res["oracle_sample"] = f"256 rays of one sensor, brute force over 1.08M Gaussians, FP64, {os.cpu_count()} cores"
    return res


def mesh_leg(dev, warmup, steps):
    """Mesh -> Gaussian transfer of a 1M-facet coloured heightfield into SH-degree-3 node
    arrays.  HBM-bound: algorithmic bytes = 12 B of indices per facet, every vertex position
    and colour read once (24 B per vertex), 236 B written per facet."""
    import numpy as np
    import torch
    from paper_2507_21981_gb300 import dgs as D
    from paper_2507_21981_gb300 import scenes
    from paper_2507_21981_gb300.render import Renderer
    v, f, col = scenes.mesh_heightfield(5, 708, 708, size=4.0, amp=0.2)
    dv, df, dc = (torch.as_tensor(a).to(dev) for a in (v, f, col))
    F = len(f)
    out = [torch.empty((F, 3), device=dev), torch.empty((F, 3), device=dev), torch.empty((F, 4), device=dev),
           torch.empty((F,), device=dev), torch.empty((F, 16, 3), device=dev)]
    r = Renderer()
    stream = torch.cuda.current_stream(dev)

    def call():
        rc = D.dgs_mesh_to_gaussians(r.ctx, dv, len(v), df, F, dc, 0.01, 2.0, 3, *out, stream.cuda_stream)
        assert rc == D.DGS_OK
    for _ in range(warmup):
        call()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(steps):
        call()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / steps
    r.close()
    # the kernel alone: CUDA events recorded by the library around it (profile = 1)
    rp = Renderer(profile=1)
    kms = []
    for _ in range(steps):
        rc = D.dgs_mesh_to_gaussians(rp.ctx, dv, len(v), df, F, dc, 0.01, 2.0, 3, *out, stream.cuda_stream)
        assert rc == D.DGS_OK
        kms.append(rp.kernel_times()["mesh"])
    rp.close()
    k_ms = float(np.median(kms))
    byt = F * (12 + 236) + len(v) * 24
    peaks, kind = _peaks()
    # the oracle on a sample of the facets (numpy FP64)
    import oracle
    idx = np.arange(20_000)
    t0 = time.perf_counter()
    oracle.mesh.mesh_to_gaussians(v, f[idx], vertex_colors=col, sh_degree=3)
    t_or = time.perf_counter() - t0
    return {"workload": "1M-facet coloured heightfield (708 x 708 vertices) -> SH3 Gaussian node", "facets": F,
            "ms_per_call": ms, "mfacets_s": F / ms / 1e3, "kernel_ms": k_ms,
            "roofline": {"bound": "hbm", "bytes": byt, "achieved": byt / k_ms / 1e6, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": byt / k_ms / 1e6 / peaks["hbm_gbs"],
                         "peak_source": f"{kind} MEASURED_PEAKS.json hbm_gbs"},
            "note": "ms_per_call includes the call's stream synchronisation; kernel_ms is the kernel alone",
            "oracle_mfacets_s": 20_000 / t_or / 1e6, "oracle_sample": "20k facets, numpy FP64, 1 thread", "steps": steps}


def tsdf_leg(dev, sc, warmup, steps):
    """Gaussian node -> mesh, first half (Sec. III-B): 64 depth views of env 0 of the benchmark
    scene (room + objects) from a ring of cameras around the workspace, rendered by the library,
    then fused into a 256^3 TSDF over a 1.2 m cube around the workspace (4.7 mm voxels).  The
    fusion kernel is timed with the library's CUDA events; its work is 16.8M voxels x 64 views."""
    import numpy as np
    import torch
    from paper_2507_21981_gb300 import dgs as D
    from paper_2507_21981_gb300 import scenes
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    c = scenes.WORKSPACE_CENTRE
    cams = []
    for k in range(64):
        az = 2 * np.pi * k / 64
        el = np.deg2rad(20 + 25 * (k % 2))
        eye = c + 1.1 * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        cams.append((500.0, 500.0, 320.0, 240.0, 640, 480, scenes.look_at(eye, c)))
    ks = [int(x) for x in sc.env_node_ids[0] if x >= 0]
    one = scenes.scene_from_lists("tsdf", sc.nodes, [ks], [[sc.node_poses[0, j] for j in range(len(ks))]], [cams])
    ds = DeviceScene(one, device=dev, spatial_order=True)
    r = Renderer(mode="batched")
    rgb, depth, alpha = r.render(ds)
    n, side = 256, 1.2
    origin = (c - side / 2).astype(np.float32)
    F = torch.zeros((n, n, n), device=dev)
    W = torch.zeros((n, n, n), device=dev)
    cam_arr = D.cameras(cams)
    rp = Renderer(profile=1)
    stream = torch.cuda.current_stream(dev)
    kms = []
    for it in range(warmup + steps):
        F.zero_(); W.zero_()
        rc = D.dgs_tsdf_integrate(rp.ctx, F, W, n, n, n, origin, side / n, 0.02, 100.0, 0.5, cam_arr, 64, depth, alpha,
                                  None, stream.cuda_stream)
        assert rc == D.DGS_OK
        if it >= warmup:
            kms.append(rp.kernel_times()["tsdf"])
    rp.close()
    r.close()
    k_ms = float(np.median(kms))
    upd = n ** 3 * 64
    seen = float((W > 0).float().mean())
    mhz = _peaks()[0].get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = n_sm * 128 * mhz * 1e6 / 1e12
    ops = upd * TSDF_OPS
    res = {"workload": "64 rendered depth views (640x480) of env 0 -> 256^3 TSDF over a 1.2 m cube", "voxels": n ** 3,
           "views": 64, "kernel_ms": k_ms, "gupdates_s": upd / k_ms / 1e6, "observed_frac": seen,
           "roofline": {"bound": "alu", "achieved": ops / k_ms / 1e9, "peak": peak, "unit": "Tops/s FP32",
                        "frac": ops / k_ms / 1e9 / peak, "ops_per_voxel_view": TSDF_OPS,
                        "peak_source": f"{n_sm} SMs (device properties) x 128 FP32 lanes x max SM clock"},
           "steps": steps}
    # the oracle on a 24^3 block of the grid (numpy FP64, one thread)
    import oracle
    Dh = depth.cpu().numpy().reshape(64, 480, 640)
    Ah = alpha.cpu().numpy().reshape(64, 480, 640)
    t0 = time.perf_counter()
    oracle.tsdf.integrate(np.zeros((24, 24, 24)), np.zeros((24, 24, 24)), origin.astype(np.float64) + 0.5, side / n,
                          0.02, 100.0, 0.5, cams, Dh, Ah)
    dt = time.perf_counter() - t0
    res["oracle_gupdates_s"] = 24 ** 3 * 64 / dt / 1e9
    res["oracle_sample"] = "24^3 voxels x 64 views, numpy FP64, 1 thread"
    return res


def _oracle_workload(seed=1):
    """The benchmark workload (config 2) and its FP64 copy for the oracle, built once."""
    import oracle
    from paper_2507_21981_gb300 import scenes
    sc = scenes.config2(seed=seed)
    return sc, oracle.oracle._Packed(sc)


def cpu_baseline(views=1, seed=1, first=0, workload=None):
    """Times the FP64 oracle on `views` sampled views of the workload (host cores): views
    first, first + 1, ... of a fixed spread over envs and both camera kinds."""
    import oracle
    sc, pk = workload or _oracle_workload(seed)
    opts = oracle.OracleOptions()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    px = 0
    for v in range(first, first + views):
        e, c = sc.views[(v * 37) % sc.n_views]     # spread over envs and both camera kinds
        r = oracle.render_view(sc, e, c, opts, pk)
        px += r.depth.size
    dt = time.perf_counter() - t0
    return {"value": px / dt / 1e6, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
            "sample": f"{views} view(s) of the workload, 640x480, full 1.08M-Gaussian scene, FP64, {dt:.1f} s"}


def oracle_timings():
    """The FP64 oracle timed per configuration on the host cores (all threads unless stated):
    config 1 every view, configs 3 and 5 on seeded sampled views (2 for config 5: its 3.3M
    Gaussians per view make each view slow), config 4 forward + backward of its one view, and
    one config-2 view on a single thread."""
    import numpy as np
    import oracle
    from paper_2507_21981_gb300 import scenes
    res = {"cores": os.cpu_count()}
    rng = np.random.default_rng(2)

    def views(sc, idx, opts=None):
        pk = oracle.oracle._Packed(sc)
        t0 = time.perf_counter()
        px = 0
        for v in idx:
            e, c = sc.views[int(v)]
            px += oracle.render_view(sc, e, c, opts or oracle.OracleOptions(), pk).depth.size
        dt = time.perf_counter() - t0
        return {"mpix_s": px / dt / 1e6, "views": [int(v) for v in idx], "seconds": dt}
    sc = scenes.config1(seed=1)
    res["config1"] = views(sc, range(sc.n_views))
    sc = scenes.config3(seed=1)
    res["config3"] = views(sc, rng.choice(sc.n_views, 4, replace=False))
    sc = scenes.config5(seed=1)
    res["config5"] = views(sc, rng.choice(sc.n_views, 2, replace=False))
    sc = scenes.config2(seed=1)
    res["config2_single_thread"] = views(sc, [0], oracle.OracleOptions(nthreads=1))
    sc = scenes.config4(seed=1)
    pk = oracle.oracle._Packed(sc)
    g = np.random.default_rng(0).normal(size=(800, 800, 3))
    gd = np.random.default_rng(1).normal(size=(800, 800))
    t0 = time.perf_counter()
    oracle.render_view(sc, 0, 0, oracle.OracleOptions(), pk)
    oracle.backward_view(sc, 0, 0, g, gd, oracle.OracleOptions(), pk)
    res["config4_fwd_bwd_ms"] = (time.perf_counter() - t0) * 1e3
    return res


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    wl = _oracle_workload(1)                   # built once, outside every step
    for i in range(args.warmup):               # untimed: first touches of the scene's pages
        cpu_baseline(views=1, first=i, workload=wl)
    samples = [cpu_baseline(views=1, first=args.warmup + i, workload=wl) for i in range(args.steps)]
    val = statistics.median(s["value"] for s in samples)
    cb = dict(samples[0]); cb["value"] = val
    cb["sample"] = f"1 view per step ({args.steps} different views), 640x480, full 1.08M-Gaussian scene, FP64"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "1 view per step, a different view each step"},
            "cpu_baseline": cb, "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--envs", type=int, default=64, help="envs per rank (64 = the benchmark workload)")
    ap.add_argument("--only-batched", action="store_true",
                    help="time the batched render only (no e2e, plain or CPU legs): small profiling runs")
    ap.add_argument("--no-extra", action="store_true", help="skip the ragged and precision workloads")
    ap.add_argument("--only-leg", choices=["augment", "lidar", "mesh", "tsdf", "fwd_bwd", "render"], default=None,
                    help="run one side workload alone on --envs envs and print its JSON (profiling runs); "
                         "'render' renders the batch --renders times with the tile shape --tile as one view group")
    ap.add_argument("--tile", default="16x16", help="tile shape of --only-leg render")
    ap.add_argument("--renders", type=int, default=2, help="renders of --only-leg render")
    ap.add_argument("--views-per-group", type=int, default=0,
                    help="views per group of the batched sequence (0 = as few groups as the sort allows)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2507_21981_gb300.render import DeviceScene, Renderer

    sc = rank_scene(rank, args.envs)
    ds = DeviceScene(sc, device=dev, spatial_order=True)
    if args.only_leg:
        if args.only_leg == "augment":
            o = (torch.empty((ds.n_pixels, 3), device=dev), torch.empty((ds.n_pixels,), device=dev), None)
            res = augment_leg(dev, ds, (16, 16), o, args.warmup, args.steps, float("nan"))
        elif args.only_leg == "lidar":
            res = lidar_leg(dev, ds, args.warmup, args.steps)
        elif args.only_leg == "mesh":
            res = mesh_leg(dev, args.warmup, args.steps)
        elif args.only_leg == "fwd_bwd":
            res = fwd_bwd_500k(dev, args.warmup, args.steps)
        elif args.only_leg == "render":
            tw, th = (int(x) for x in args.tile.split("x"))
            rr = Renderer(mode="batched", tile=(tw, th), views_per_group=ds.n_views)
            for _ in range(args.renders):
                rr.render(ds)
            torch.cuda.synchronize(dev)
            res = {"tile": args.tile, "renders": args.renders, "stats": rr.stats()}
            rr.close()
        else:
            res = tsdf_leg(dev, sc, args.warmup, args.steps)
        if rank == 0:
            print(json.dumps({"leg": args.only_leg, **res}))
        return 0
    stream = torch.cuda.current_stream(dev)
    px_per_step = ds.n_pixels

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # ---------------------------------------------------------------- batched, resident inputs
    out = (torch.empty((px_per_step, 3), device=dev), torch.empty((px_per_step,), device=dev),
           torch.empty((px_per_step,), device=dev))
    # the tile shape for this workload, picked by the library's autotuner (outside the timed region)
    vpg = args.views_per_group
    tuner = Renderer(mode="batched", views_per_group=vpg)
    tile, tile_ms, _ = tuner.autotune(ds, reps=2, out=out)
    tuner.close()
    # headline: the default sequence (a large batch runs as two pipelined view groups), no
    # per-kernel events
    rb = Renderer(mode="batched", tile=tile, views_per_group=vpg)
    launches = 0
    with ClockSampler(local) as clk:            # started before the warm-up: nvidia-smi takes a moment
        for _ in range(args.warmup):
            rb.render(ds, out=out)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        clk.mark_start()
        ev0.record(stream)
        for _ in range(args.steps):
            rb.render(ds, out=out)
            launches += rb.launches()
        ev1.record(stream)
        barrier()
        clk.mark_end()
    ms = ev0.elapsed_time(ev1) / args.steps
    groups = rb.stats()["n_groups"]
    # per-kernel breakdown: the same batch as one view group (kernels not overlapped), CUDA
    # events recorded by the library around each kernel class on the launching stream
    rk = Renderer(mode="batched", tile=tile, profile=True, views_per_group=ds.n_views)
    for _ in range(args.warmup):
        rk.render(ds, out=out)
    ktimes = {k: 0.0 for k in rk.kernel_times()}
    ek0, ek1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ek0.record(stream)
    for _ in range(args.steps):
        rk.render(ds, out=out)
        for k, v in rk.kernel_times().items():
            ktimes[k] += v
    ek1.record(stream)
    barrier()
    ms_one_group = ek0.elapsed_time(ek1) / args.steps
    stats = rk.stats()
    rk.close()
    if args.only_batched:
        if rank == 0:
            print(json.dumps({"value_mpix_s": px_per_step / (ms / 1e3) / 1e6, "ms_per_step": ms, "envs": args.envs,
                              "kernel_ms_per_step": {k: v / args.steps for k, v in ktimes.items()},
                              "render_stats": stats}))
        return 0
    ms = max_over_ranks(ms, world, dev)
    value = px_per_step * world / (ms / 1e3) / 1e6

    # ---------------------------------------------------------------- the same batch as graph replays
    rg = Renderer(mode="graph", tile=tile)
    for _ in range(args.warmup):
        rg.render(ds, out=out)
    barrier()
    ms_graph = max_over_ranks(_time_renders(rg, ds, out, args.steps, stream), world, dev)
    graph_path = rg.stats()["path"]
    graph_value = px_per_step * world / (ms_graph / 1e3) / 1e6
    rg.close()

    # ---------------------------------------------------------------- e2e through the C ABI with host buffers
    # every step uploads its poses from pinned host memory and reads its RGB + depth back into
    # pinned host memory.  Two host threads each drive their own graph-mode context, stream,
    # output buffers and pinned buffers (a context belongs to one thread at a time), so while
    # one thread's call waits for its render the other stages and launches the next step: two
    # steps are in flight, and each step's read-back runs on its thread's copy stream while the
    # next renders.  The timed region starts on an event that both streams wait for and ends
    # after the last read-back of both.
    import copy as _copy
    poses_np = np.ascontiguousarray(sc.node_poses, np.float32).reshape(ds.n_envs, ds.max_nodes, 12)
    n_workers = 2
    per_worker = (args.steps + n_workers - 1) // n_workers
    e2e_steps = per_worker * n_workers
    workers = []
    for w in range(n_workers):
        dsw = _copy.copy(ds)                     # shares the scene's tensors; own pose buffer
        dsw.node_poses = torch.empty_like(ds.node_poses)
        workers.append({
            "ds": dsw, "r": Renderer(mode="graph", tile=tile), "s": torch.cuda.Stream(dev),
            "cs": torch.cuda.Stream(dev), "poses": torch.from_numpy(poses_np.copy()).pin_memory(),
            "host": (torch.empty((px_per_step, 3), dtype=torch.float32).pin_memory(),
                     torch.empty((px_per_step,), dtype=torch.float32).pin_memory()),
            "dev": ((out[0], out[1]) if w == 0 else
                    (torch.empty_like(out[0]), torch.empty_like(out[1]))),
            "copied": torch.cuda.Event(), "spans": []})

    def e2e_step(w):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(w["s"]):
            w["ds"].node_poses.copy_(w["poses"], non_blocking=True)
        w["s"].wait_event(w["copied"])           # this worker's previous read-back is done
        ev[0].record(w["s"])
        rgb, depth, _ = w["r"].render(w["ds"], out=(w["dev"][0], w["dev"][1], None), stream=w["s"])
        ev[1].record(w["s"])
        w["cs"].wait_event(ev[1])
        with torch.cuda.stream(w["cs"]):
            ev[2].record(w["cs"])
            w["host"][0].copy_(rgb, non_blocking=True)
            w["host"][1].copy_(depth, non_blocking=True)
            ev[3].record(w["cs"])
        w["copied"].record(w["cs"])
        w["spans"].append(ev)

    for _ in range(args.warmup):                 # captures the graphs one context at a time
        for w in workers:
            e2e_step(w)
    barrier()
    for w in workers:
        w["spans"].clear()
    ev0.record(stream)
    for w in workers:
        w["s"].wait_event(ev0)
    errors = []
    start = threading.Barrier(n_workers)         # both host threads start their steps together

    def run_worker(w):
        try:
            start.wait()
            for _ in range(per_worker):
                e2e_step(w)
        except Exception as exc:                 # reported after the join
            errors.append(exc)
    threads = [threading.Thread(target=run_worker, args=(w,)) for w in workers]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    for w in workers:
        stream.wait_event(w["copied"])
        stream.wait_stream(w["s"])
    ev1.record(stream)
    barrier()
    host_rgb, host_depth = workers[0]["host"]
    ms_e2e = max_over_ranks(ev0.elapsed_time(ev1) / e2e_steps, world, dev)
    spans = [e for w in workers for e in w["spans"]]
    e2e_render_ms = float(np.median([e[0].elapsed_time(e[1]) for e in spans]))
    e2e_copy_ms = float(np.median([e[2].elapsed_time(e[3]) for e in spans]))
    for w in workers:
        w["r"].close()
    e2e_value = px_per_step * world / (ms_e2e / 1e3) / 1e6
    h2d = poses_np.nbytes
    d2h = (host_rgb.numel() + host_depth.numel()) * 4

    # ---------------------------------------------------------------- plain per-view FP32 (same scene, same GPU)
    rp = Renderer(mode="plain")
    for _ in range(2):
        rp.render(ds, out=out)
    barrier()
    ev0.record(stream)
    for _ in range(args.plain_steps):
        rp.render(ds, out=out)
    ev1.record(stream)
    barrier()
    ms_plain = max_over_ranks(ev0.elapsed_time(ev1) / args.plain_steps, world, dev)
    plain_value = px_per_step * world / (ms_plain / 1e3) / 1e6
    rp.close()
    # the plain form's projection passes, timed by the library's events (one call)
    rpp = Renderer(mode="plain", profile=True)
    rpp.render(ds, out=out)
    plain_k = rpp.kernel_times()
    plain_stats = rpp.stats()
    rpp.close()

    # ---------------------------------------------------------------- fwd+bwd at 500k Gaussians (one 800x800 view)
    fb = fwd_bwd_500k(dev, args.warmup, max(3, args.steps // 4))
    extra = {}
    if not args.no_extra and world == 1:       # single-GPU workloads, reported at N = 1
        extra["ragged"] = ragged_graph(dev, args.warmup, max(3, args.steps // 4))
        extra["precision_scale"] = precision_scale(dev, args.warmup, max(3, args.steps // 4))
        extra["augment"] = augment_leg(dev, ds, tile, out, args.warmup, max(3, args.steps // 4), ms)
        extra["lidar"] = lidar_leg(dev, ds, args.warmup, max(3, args.steps // 8))
        extra["mesh"] = mesh_leg(dev, args.warmup, max(3, args.steps // 4))
        extra["tsdf"] = tsdf_leg(dev, sc, args.warmup, max(3, args.steps // 8))

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    # ---------------------------------------------------------------- roofline of the dominant kernel class
    peaks, peak_kind = _peaks()
    per_step = {k: v / args.steps for k, v in ktimes.items()}
    dom = max(per_step, key=per_step.get)
    P, NV = stats["n_pairs"], stats["n_visible"]
    passes = (stats["key_bits"] + 7) // 8          # tile-sort passes (key_bits = tile key bits)
    # passes of the depth sort's view key (the bits of the views per group; none for one view);
    # the view rides in the instance numbers' high bits when both fit in 32 bits, else each
    # view pass also gathers the view of every value (4 B)
    vpg = -(-stats["n_views"] // max(stats["n_groups"], 1))
    vbits = (vpg - 1).bit_length()
    vpasses = (vbits + 7) // 8
    packed = vbits > 0 and (max(NV // max(stats["n_groups"], 1), 1) - 1).bit_length() + vbits <= 32
    # algorithmic bytes of the binning class: depth sort of the instances (28-bit keys: the
    # histogram read, 4 passes of 16 B, the last writing no keys when view passes follow; each
    # view pass reads and writes the value), tile-count scan (order and count read twice, offset
    # written: 20 B), pair emission (record 48 + identity 8 + order 4 + offset 4 read; 8 B
    # written per pair) and the tile sort (histogram read, passes of 16 B)
    depth_b = 4 + 4 * 16 - (4 if vpasses else 0) + vpasses * (8 if packed else 12)
    sort_bytes = NV * (depth_b + 20 + 64) + P * (8 + 4 + passes * 16)
    # compositor work of one step, counted by the instrumented compositor outside the timed region
    rc_ = Renderer(mode="batched", tile=tile, profile=2)
    rc_.render(ds, out=out)
    work = rc_.stats()
    rc_.close()
    mhz = peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * 128 * mhz * 1e6 / 1e12         # FP32 lane-ops per second (FMA counted once), T/s
    alu_src = f"{n_sm} SMs (device properties) x 128 FP32 lanes x max SM clock {mhz:.0f} MHz ({peak_kind} MEASURED_PEAKS.json)"
    hbm_src = f"{peak_kind} MEASURED_PEAKS.json hbm_gbs"
    alu = lambda ops, ms_: {"bound": "alu", "unit": "Tops/s FP32", "peak": fp32_peak, "peak_source": alu_src,
                            "achieved": ops / (ms_ / 1e3) / 1e12}
    hbm = lambda byt, ms_: {"bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"], "peak_source": hbm_src,
                            "achieved": byt / (ms_ / 1e3) / 1e9}
    comp_ops = work["px_reached"] * OPS_PER_PAIR
    n_inst = stats["n_instances"]
    kernels = {
        "composite": {**alu(comp_ops, per_step["composite"]),
                      "units": {"pairs_reached": work["px_reached"], "pairs_composited": work["px_composited"],
                                "pairs_evaluated": work["px_evaluated"],
                                "evaluated_over_reached": work["px_evaluated"] / max(work["px_reached"], 1),
                                "ops_per_pair": OPS_PER_PAIR}},
        "sort": {**hbm(sort_bytes, per_step["sort"]),
                 "units": {"instances": NV, "pairs": P, "depth_passes": 4, "view_passes": vpasses,
                           "view_key": "packed in the values" if packed else "gathered",
                           "tile_passes": passes, "bytes_per_instance": depth_b + 20 + 64,
                           "bytes_per_pair": 8 + 4 + passes * 16}},
        "emit": {**alu(NV * (PROJ_OPS + SH3_OPS), per_step["emit"]),
                 "units": {"visible": NV, "ops_per_visible": PROJ_OPS + SH3_OPS,
                           "not_counted": "tile-row runs of the pair count"}},
        "count": {**alu(NV * CULL_OPS, per_step["count"]),
                  "units": {"visible": NV, "ops_per_visible": CULL_OPS,
                            "not_counted": "chunk and per-Gaussian culls",
                            "instances_considered": n_inst}},
        # the plain per-view form reads every attribute again for every view
        "plain_projection": {**hbm(n_inst * (40 + 236) + plain_stats["n_visible"] * 68,
                                   plain_k["count"] + plain_k["emit"]),
                             "units": {"instances": n_inst, "bytes_per_instance": 40 + 236,
                                       "visible": plain_stats["n_visible"], "bytes_per_visible": 68,
                                       "ms": plain_k["count"] + plain_k["emit"]}},
    }
    fk, fw = fb.get("kernel_ms", {}), fb.get("work", {})
    if fk.get("bwd_backward") and fk.get("bwd_backward_project"):
        kernels["composite_bwd"] = {**alu(fw["pairs_composited"] * BWD_OPS_PER_PAIR, fk["bwd_backward"]),
                                    "units": {"pairs_composited": fw["pairs_composited"],
                                              "ops_per_pair": BWD_OPS_PER_PAIR,
                                              "reductions": fw["bwd_reductions"],
                                              "reductions_per_s": fw["bwd_reductions"] / (fk["bwd_backward"] / 1e3),
                                              "workload": "800x800 view, 500k Gaussians"}}
        kernels["project_bwd"] = {**hbm(fw["visible"] * PROJECT_BWD_BYTES, fk["bwd_backward_project"]),
                                  "units": {"visible": fw["visible"], "bytes_per_visible": PROJECT_BWD_BYTES,
                                            "workload": "800x800 view, 500k Gaussians"}}
    for k in kernels.values():
        k["frac"] = k["achieved"] / k["peak"]
    dk = dom if dom in kernels else "composite"
    d = kernels[dk]
    roof = {"kernel": dk, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
            "frac": d["frac"], "traffic": TRAFFIC.get(dk), "peak_source": d["peak_source"]}
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "sm_count": n_sm,
        "data": "synthetic (seeded room + objects; the paper's scanned scenes are not available)",
        "config": {"workload": WORKLOAD, "views": ds.n_views, "pixels_per_step": px_per_step, "gaussians": sc.n_gaussians,
                   "l2": "inputs larger than L2 (255 MB attributes, 629 MB outputs per step)", "mode": "batched",
                   "tile": f"{tile[0]}x{tile[1]}", "autotune_ms": {f"{w}x{h}": t for (w, h), t in tile_ms.items()},
                   "layout": "nodes stored in Z-order of their means (dgs_spatial_order, once at load)"},
        "plain_mpix_s": plain_value, "batched_over_plain": value / plain_value,
        "graph_mpix_s": graph_value, "graph_path": graph_path,
        "fwd_bwd_ms_per_view_500k": fb["ms"],
        "fwd_bwd_detail": fb,
        "view_groups": groups, "one_group_mpix_s": px_per_step * world / (ms_one_group / 1e3) / 1e6,
        "kernel_ms_per_step": per_step, "kernel_times_from": "one-view-group profiled region (kernels not overlapped)",
        "render_stats": stats,
        "roofline": roof, "kernel_rooflines": kernels,
        "e2e": {"value": e2e_value, "unit": "Mpix/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": ms_e2e, "steps": e2e_steps, "render_ms_median": e2e_render_ms,
                "readback_ms_median": e2e_copy_ms,
                "note": "two host threads, each with its own context, stream and buffers, keep two steps in "
                        "flight; a step's render span overlaps the other thread's step"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    line.update(extra)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(views=16)
        if world == 1:
            line["oracle_timing"] = oracle_timings()
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
