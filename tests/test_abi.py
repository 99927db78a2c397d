"""The C-ABI library loads, exports every function include/dgs.h declares, and validates
arguments on the host (no GPU needed: only calls that return before any device work)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2507_21981_gb300 import build as B
from paper_2507_21981_gb300 import dgs as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(dgs_\w+)\s*\(", src, re.M)
    return sorted(set(names))


def test_header_declares_the_render_calls():
    names = declared_functions()
    for n in ("dgs_render", "dgs_context_create", "dgs_context_destroy", "dgs_last_error"):
        assert n in names


def test_every_declared_function_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_covers_every_export(lib):
    for n in declared_functions():
        assert n in D.EXPORTED, n


def test_default_options(lib):
    o = D.dgs_default_options()
    assert (o.tile_w, o.tile_h, o.mode) == (16, 16, D.DGS_MODE_BATCHED)
    assert o.alpha_min == pytest.approx(1 / 255) and o.alpha_max == pytest.approx(0.99)
    assert o.t_min == pytest.approx(1e-4) and o.q_max == 9.0 and o.lowpass == pytest.approx(0.3)
    assert o.z_near == pytest.approx(0.01) and o.guard == pytest.approx(1.3)


def test_struct_sizes_match_header(lib):
    assert C.sizeof(D.dgs_node) == 56
    assert C.sizeof(D.dgs_camera) == 72
    assert C.sizeof(D.dgs_options) == 80
    assert C.sizeof(D.dgs_stats) == 88
    assert C.sizeof(D.dgs_tune_result) == 8 + 3 * 4 * D.DGS_TUNE_MAX
    assert C.sizeof(D.dgs_augment) == 32
    assert C.sizeof(D.dgs_lidar) == 52


def test_augment_record_layout_matches_the_numpy_generator():
    from paper_2507_21981_gb300 import scenes as S
    assert S.AUGMENT_DTYPE.itemsize == C.sizeof(D.dgs_augment)
    for name, _ in D.dgs_augment._fields_:
        assert S.AUGMENT_DTYPE.fields[name][1] == getattr(D.dgs_augment, name).offset, name


def test_invalid_options_rejected(lib):
    o = D.dgs_default_options()
    o.tile_w = 10
    h = C.c_void_p()
    assert lib.dgs_context_create(C.byref(h), C.byref(o)) == D.DGS_ERR_INVALID_ARG
    o = D.dgs_default_options()
    o.z_near = 0.0
    assert lib.dgs_context_create(C.byref(h), C.byref(o)) == D.DGS_ERR_INVALID_ARG
    assert lib.dgs_context_create(None, None) == D.DGS_ERR_INVALID_ARG


def _ctx(lib):
    h = C.c_void_p()
    assert lib.dgs_context_create(C.byref(h), None) == D.DGS_OK
    return h


def _args(n_nodes=1, E=1, K=1, Cm=1):
    nodes = (D.dgs_node * n_nodes)()
    for k in range(n_nodes):
        nodes[k].n = 0
        nodes[k].sh_degree = 0
        nodes[k].dtype = D.DGS_F32
    ids = np.zeros((E, K), np.int32)
    cams = (D.dgs_camera * (E * Cm))()
    for i in range(E * Cm):
        cams[i].fx = cams[i].fy = 10.0
        cams[i].width = cams[i].height = 8
        cams[i].cam_from_world[:] = [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]
    cpe = np.ones(E, np.int32)
    return nodes, ids, cams, cpe


FAKE_DEV = 0x10000   # never dereferenced: every case below fails host validation first


def _render(lib, ctx, nodes, n_nodes, ids, E, K, cams, cpe, Cm, poses=FAKE_DEV, rgb=FAKE_DEV, depth=FAKE_DEV):
    return lib.dgs_render(ctx, nodes, n_nodes, ids.ctypes.data, E, K, poses, cams, cpe.ctypes.data, Cm, rgb, depth,
                          None, None, None)


def test_render_validates_arguments_on_host(lib):
    ctx = _ctx(lib)
    try:
        nodes, ids, cams, cpe = _args()
        assert lib.dgs_render(None, nodes, 1, ids.ctypes.data, 1, 1, FAKE_DEV, cams, cpe.ctypes.data, 1, FAKE_DEV,
                              FAKE_DEV, None, None, None) == D.DGS_ERR_INVALID_ARG
        # missing outputs
        assert _render(lib, ctx, nodes, 1, ids, 1, 1, cams, cpe, 1, rgb=None) == D.DGS_ERR_INVALID_ARG
        assert "out_rgb" in D.dgs_last_error(ctx)
        # node id out of range / duplicated in one env
        bad = ids.copy(); bad[0, 0] = 5
        assert _render(lib, ctx, nodes, 1, bad, 1, 1, cams, cpe, 1) == D.DGS_ERR_INVALID_ARG
        n2, ids2, cams2, cpe2 = _args(n_nodes=1, K=2)
        assert _render(lib, ctx, n2, 1, ids2, 1, 2, cams2, cpe2, 1) == D.DGS_ERR_INVALID_ARG
        assert "twice" in D.dgs_last_error(ctx)
        # bad SH degree and dtype
        nodes[0].sh_degree = 4
        assert _render(lib, ctx, nodes, 1, ids, 1, 1, cams, cpe, 1) == D.DGS_ERR_INVALID_ARG
        nodes[0].sh_degree = 0; nodes[0].dtype = 7
        assert _render(lib, ctx, nodes, 1, ids, 1, 1, cams, cpe, 1) == D.DGS_ERR_INVALID_ARG
        nodes[0].dtype = 0
        # a non-empty node with null attribute pointers
        nodes[0].n = 10
        assert _render(lib, ctx, nodes, 1, ids, 1, 1, cams, cpe, 1) == D.DGS_ERR_INVALID_ARG
        nodes[0].n = 0
        # camera: non-rigid rotation, non-positive focal length, zero size, too many cameras
        cams[0].cam_from_world[0] = 2.0
        assert _render(lib, ctx, nodes, 1, ids, 1, 1, cams, cpe, 1) == D.DGS_ERR_INVALID_ARG
        cams[0].cam_from_world[0] = 1.0; cams[0].fx = -1.0
        assert _render(lib, ctx, nodes, 1, ids, 1, 1, cams, cpe, 1) == D.DGS_ERR_INVALID_ARG
        cams[0].fx = 10.0; cams[0].width = 0
        assert _render(lib, ctx, nodes, 1, ids, 1, 1, cams, cpe, 1) == D.DGS_ERR_INVALID_ARG
        cams[0].width = 8
        cpe[0] = 2
        assert _render(lib, ctx, nodes, 1, ids, 1, 1, cams, cpe, 1) == D.DGS_ERR_INVALID_ARG
        cpe[0] = 1
        cams[0].cam_from_world[3] = float("nan")
        assert _render(lib, ctx, nodes, 1, ids, 1, 1, cams, cpe, 1) == D.DGS_ERR_INVALID_ARG
    finally:
        lib.dgs_context_destroy(ctx)


def test_graph_mode_is_accepted_and_bad_modes_rejected(lib):
    o = D.dgs_default_options()
    o.mode = D.DGS_MODE_GRAPH
    h = C.c_void_p()
    assert lib.dgs_context_create(C.byref(h), C.byref(o)) == D.DGS_OK
    lib.dgs_context_destroy(h)
    o.mode = 3
    assert lib.dgs_context_create(C.byref(h), C.byref(o)) == D.DGS_ERR_INVALID_ARG


def test_autotune_validates_arguments_on_host(lib):
    ctx = _ctx(lib)
    try:
        nodes, ids, cams, cpe = _args()
        res = D.dgs_tune_result()

        def tune(cand, nc, reps, out=True):
            cp = None if cand is None else np.ascontiguousarray(np.asarray(cand, np.int32)).ctypes.data
            return lib.dgs_autotune(ctx, nodes, 1, ids.ctypes.data, 1, 1, FAKE_DEV, cams, cpe.ctypes.data, 1,
                                    FAKE_DEV, FAKE_DEV, None, None, cp, nc, reps, C.byref(res) if out else None, None)
        assert tune(None, 0, 3, out=False) == D.DGS_ERR_INVALID_ARG
        assert tune(None, 0, 0) == D.DGS_ERR_INVALID_ARG                  # reps
        assert tune([[16, 16]] * 17, 17, 1) == D.DGS_ERR_INVALID_ARG      # too many candidates
        assert tune([[16, 16], [12, 8]], 2, 1) == D.DGS_ERR_INVALID_ARG   # 12 is not a multiple of 8
        assert "candidate 1" in D.dgs_last_error(ctx)
        assert tune([[16, 32]], 1, 1) == D.DGS_ERR_INVALID_ARG            # area 512
    finally:
        lib.dgs_context_destroy(ctx)


def test_build_flags_target_sm103a():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _aug(n, **kw):
    from paper_2507_21981_gb300 import scenes as S
    a = np.zeros(n, S.AUGMENT_DTYPE)
    a["sat_scale"] = 1.0
    a["val_scale"] = 1.0
    a["gamma"] = 1.0
    for k, v in kw.items():
        a[k] = v
    return a


def test_set_augment_validates_on_host(lib):
    ctx = _ctx(lib)
    try:
        def setp(a, ov=None, nf=0, w=0, h=0):
            return lib.dgs_set_augment(ctx, None if a is None else a.ctypes.data, 0 if a is None else len(a), ov,
                                       nf, w, h)
        assert lib.dgs_set_augment(None, None, 0, None, 0, 0, 0) == D.DGS_ERR_INVALID_ARG
        assert setp(_aug(2)) == D.DGS_OK                                   # no overlay needed at weight 0
        assert setp(None) == D.DGS_OK                                      # clears
        assert lib.dgs_set_augment(ctx, _aug(1).ctypes.data, -1, None, 0, 0, 0) == D.DGS_ERR_INVALID_ARG
        for bad in (dict(gamma=0.0), dict(gamma=float("inf")), dict(sat_scale=-0.1), dict(val_scale=float("nan")),
                    dict(hue_shift=float("inf")), dict(overlay_beta=1.5), dict(overlay_beta=float("nan"))):
            assert setp(_aug(2, **bad)) == D.DGS_ERR_INVALID_ARG, bad
        assert setp(_aug(2, overlay_beta=0.5)) == D.DGS_ERR_INVALID_ARG  # weight > 0 without an overlay
        assert "overlay" in D.dgs_last_error(ctx)
        assert setp(_aug(2, overlay_beta=0.5), FAKE_DEV, 2, 64, 48) == D.DGS_OK
        assert setp(_aug(2, overlay_beta=0.5, overlay_frame=2), FAKE_DEV, 2, 64, 48) == D.DGS_ERR_INVALID_ARG
        assert setp(_aug(2, overlay_beta=0.5, overlay_x=64), FAKE_DEV, 2, 64, 48) == D.DGS_ERR_INVALID_ARG
        assert setp(_aug(2, overlay_beta=0.5, overlay_y=-1), FAKE_DEV, 2, 64, 48) == D.DGS_ERR_INVALID_ARG
        assert setp(_aug(2), FAKE_DEV, 0, 64, 48) == D.DGS_ERR_INVALID_ARG   # bad overlay shape
        # the last valid setting (2 views) stands: a one-view render is refused before any device work
        nodes, ids, cams, cpe = _args()
        assert _render(lib, ctx, nodes, 1, ids, 1, 1, cams, cpe, 1) == D.DGS_ERR_INVALID_ARG
        assert "2 views" in D.dgs_last_error(ctx)
        # the adjoint refuses while a randomisation is set
        assert lib.dgs_render_backward(ctx, nodes, 1, ids.ctypes.data, 1, 1, FAKE_DEV, cams, cpe.ctypes.data, 1,
                                       FAKE_DEV, FAKE_DEV, FAKE_DEV, None, None, None, None, None) \
            == D.DGS_ERR_UNSUPPORTED
        # the separate pass: view count and sizes are checked on the host
        sizes = np.array([[8, 8], [8, 8]], np.int32)
        assert lib.dgs_augment_rgb(ctx, FAKE_DEV, sizes.ctypes.data, None, 1, None) == D.DGS_ERR_INVALID_ARG
        assert lib.dgs_augment_rgb(ctx, None, sizes.ctypes.data, None, 2, None) == D.DGS_ERR_INVALID_ARG
        bad = np.array([[8, 8], [0, 8]], np.int32)
        assert lib.dgs_augment_rgb(ctx, FAKE_DEV, bad.ctypes.data, None, 2, None) == D.DGS_ERR_INVALID_ARG
        neg = np.array([0, -5], np.int64)
        assert lib.dgs_augment_rgb(ctx, FAKE_DEV, sizes.ctypes.data, neg.ctypes.data, 2, None) == D.DGS_ERR_INVALID_ARG
        assert setp(None) == D.DGS_OK
        assert lib.dgs_augment_rgb(ctx, FAKE_DEV, sizes.ctypes.data, None, 2, None) == D.DGS_ERR_INVALID_ARG
        assert "no randomisation" in D.dgs_last_error(ctx)
    finally:
        lib.dgs_context_destroy(ctx)


def test_lidar_validates_on_host(lib):
    ctx = _ctx(lib)
    try:
        nodes, ids, _, _ = _args()
        sens = D.lidar_sensors([0], np.eye(3, 4)[None])

        def trace(nodes=nodes, n=1, sensors=sens, ns=1, dirs=FAKE_DEV, nd=4, r0=0.05, r1=30.0, env=1):
            return lib.dgs_lidar_trace(ctx, nodes, n, ids.ctypes.data, env, 1, FAKE_DEV, sensors, ns, dirs, nd, r0, r1,
                                       FAKE_DEV, FAKE_DEV, None)
        assert trace() == D.DGS_ERR_INVALID_ARG                        # nothing built yet
        assert "dgs_lidar_build" in D.dgs_last_error(ctx)
        assert lib.dgs_lidar_build(ctx, nodes, 0, None) == D.DGS_ERR_INVALID_ARG
        bad = (D.dgs_node * 1)()
        bad[0].n, bad[0].sh_degree, bad[0].dtype = 5, 0, 0            # null attribute pointers
        assert lib.dgs_lidar_build(ctx, bad, 1, None) == D.DGS_ERR_INVALID_ARG
    finally:
        lib.dgs_context_destroy(ctx)


def test_mesh_to_gaussians_validates_on_host(lib):
    ctx = _ctx(lib)
    try:
        def call(nv=3, nf=1, flatten=0.01, op=2.0, deg=0, quat=FAKE_DEV, v=FAKE_DEV):
            return lib.dgs_mesh_to_gaussians(ctx, v, nv, FAKE_DEV, nf, None, flatten, op, deg, FAKE_DEV, FAKE_DEV,
                                             quat, FAKE_DEV, FAKE_DEV, None)
        assert lib.dgs_mesh_to_gaussians(None, FAKE_DEV, 3, FAKE_DEV, 1, None, 0.01, 2.0, 0, FAKE_DEV, FAKE_DEV,
                                         FAKE_DEV, FAKE_DEV, FAKE_DEV, None) == D.DGS_ERR_INVALID_ARG
        assert call(nf=0) == D.DGS_OK                                       # nothing to do
        for bad in (dict(nf=-1), dict(nv=-1), dict(flatten=0.0), dict(flatten=1.5), dict(op=float("nan")),
                    dict(deg=4), dict(quat=FAKE_DEV + 4), dict(v=None)):
            assert call(**bad) == D.DGS_ERR_INVALID_ARG, bad
    finally:
        lib.dgs_context_destroy(ctx)


def test_tsdf_validates_on_host(lib):
    ctx = _ctx(lib)
    try:
        cams = D.cameras([(50.0, 50.0, 16.0, 16.0, 32, 32, np.eye(3, 4))])
        org = np.zeros(3, np.float32)

        def call(n=(4, 4, 4), org=org, vox=0.01, tr=0.05, wmax=10.0, amin=0.5, nv=1, cams=cams):
            return lib.dgs_tsdf_integrate(ctx, FAKE_DEV, FAKE_DEV, n[0], n[1], n[2], org.ctypes.data if org is not None else None,
                                          vox, tr, wmax, amin, cams, nv, FAKE_DEV, FAKE_DEV, None, None)
        assert call(nv=0) == D.DGS_OK
        for bad in (dict(n=(0, 4, 4)), dict(n=(2048, 2048, 1024)), dict(org=None), dict(vox=0.0), dict(tr=-1.0),
                    dict(wmax=0.0), dict(amin=0.0), dict(amin=1.5), dict(nv=-1)):
            assert call(**bad) == D.DGS_ERR_INVALID_ARG, bad
        bad_cam = D.cameras([(50.0, 50.0, 16.0, 16.0, 0, 32, np.eye(3, 4))])
        assert call(cams=bad_cam) == D.DGS_ERR_INVALID_ARG
    finally:
        lib.dgs_context_destroy(ctx)


def test_missing_library_fails_loudly(tmp_path):
    """No silent fallback: without the built library the binding raises instead of computing."""
    with pytest.raises(RuntimeError, match="libdgs.so not found"):
        D.load(str(tmp_path / "libdgs.so"))


def test_product_never_reaches_the_oracle():
    """The library and its binding neither import, link nor compile anything under oracle/, and
    the oracle imports nothing from the product (the two share only the seeded input
    generators, which tests pass to both)."""
    pkg = os.path.join(ROOT, "paper_2507_21981_gb300")
    use = re.compile(r"^\s*(?:import\s+oracle\b|from\s+oracle\b|#\s*include\s*[<\"][^>\"]*oracle)", re.M)
    for d, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                src = open(os.path.join(d, f)).read()
                assert not use.search(src), os.path.join(d, f)
    assert all("oracle" not in s for s in B.SOURCES)
    back = re.compile(r"^\s*(?:import\s+paper_2507_21981_gb300|from\s+paper_2507_21981_gb300)", re.M)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".cpp", ".h")):
            assert not back.search(open(os.path.join(ROOT, "oracle", f)).read()), f


def test_pose_twist_validates_arguments_on_the_host(lib):
    assert lib.dgs_pose_twist_grad(None, None, -1, None, None) == D.DGS_ERR_INVALID_ARG
    assert lib.dgs_pose_twist_grad(None, None, 3, None, None) == D.DGS_ERR_INVALID_ARG
    assert lib.dgs_pose_twist_grad(None, None, 0, None, None) == D.DGS_OK      # nothing to do, no device work


def test_debug_build_exports_every_call_and_reports_itself(lib):
    dbg = D.load(B.build(debug=True))
    for n in declared_functions():
        assert hasattr(dbg, n), n
    assert lib.dgs_build_flags() == 0
    assert dbg.dgs_build_flags() == D.DGS_BUILD_DEBUG


def test_bounds_fault_hook_needs_the_debug_build(lib):
    dbg = D.load(B.build(debug=True))
    o = D.dgs_default_options()
    o.test_fault = 3
    h = C.c_void_p()
    assert lib.dgs_context_create(C.byref(h), C.byref(o)) == D.DGS_ERR_INVALID_ARG
    assert dbg.dgs_context_create(C.byref(h), C.byref(o)) == D.DGS_OK
    dbg.dgs_context_destroy(h)
    o.test_fault = 5
    assert dbg.dgs_context_create(C.byref(h), C.byref(o)) == D.DGS_ERR_INVALID_ARG
