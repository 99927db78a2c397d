"""dgs_render_noalloc, the render for callers that cannot allocate GPU memory.

Such a caller (a program whose device memory belongs to another framework's caching
allocator, a control loop that cannot afford the synchronisation of cudaMalloc/cudaFree in a
step, code certified to allocate nothing after start-up) passes its inputs and outputs and
gets the same images as dgs_render, while the library works inside its fixed 64 MiB array.
Both run the same kernels as one view group on these batches, so the images must be equal bit
for bit; one view is also held to the FP64 oracle by the parity criterion.  Calls share the
array and leave their contents in it, so the tests interleave different batches and a
rejected batch with ordinary calls.  This file is collected last on purpose: the tests must
also pass after every other test.
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_21981_gb300 import dgs as D
from paper_2507_21981_gb300 import scenes as S
from tests.parity import compare_view

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(ds, opts, stream=None, cams=None):
    n = ds.n_pixels
    out = (torch.full((n, 3), -1.0, device=ds.device), torch.full((n,), -1.0, device=ds.device),
           torch.full((n,), -1.0, device=ds.device))
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = D.dgs_render_noalloc(opts, ds.nodes, ds.n_nodes, ds.env_node_ids, ds.n_envs, ds.max_nodes, ds.node_poses,
                              ds.cams if cams is None else cams, ds.cams_per_env, ds.max_cams, *out, None,
                              s.cuda_stream)
    torch.cuda.synchronize()
    return rc, [t.cpu().numpy() for t in out]


def _render(r, ds):
    out = [t.cpu().numpy() for t in r.render(ds)]
    torch.cuda.synchronize()
    return out


def _same(a, b, what):
    for x, y, name in zip(a, b, ("rgb", "depth", "alpha")):
        assert np.array_equal(x, y), (what, name, float(np.abs(x - y).max()))


def _scene_a():
    return S.config2(seed=5, n_envs=3, n_bg=40_000, n_obj=1_500, width=160, height=120, f=125.0)


def _scene_b():
    # fewer envs, another resolution and other poses than scene a
    return S.config2(seed=9, n_envs=2, n_bg=25_000, n_obj=1_000, width=96, height=64, f=75.0)


def test_noalloc_equals_render_bitwise_across_interleaved_batches():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    da, db = DeviceScene(_scene_a(), device="cuda:0"), DeviceScene(_scene_b(), device="cuda:0")
    r = Renderer(mode="batched")
    ref_a, ref_b = _render(r, da), _render(r, db)
    moved = []
    for call, (ds, ref) in enumerate([(da, ref_a), (db, ref_b), (da, ref_a)]):
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc, got = _noalloc(ds, r.options)
        moved.append(free_before - torch.cuda.mem_get_info()[0])
        assert rc == D.DGS_OK, D.STATUS_NAMES.get(rc, rc)
        _same(got, ref, call)
    # the output buffers are the only device memory taken; the library adds none after the first call
    n_out = [ds.n_pixels * 5 * 4 for ds in (da, db, da)]
    assert all(m <= n + (2 << 20) for m, n in zip(moved[1:], n_out[1:])), moved
    r.close()


def test_noalloc_view_against_the_oracle():
    from paper_2507_21981_gb300.render import DeviceScene
    sc = _scene_b()
    ds = DeviceScene(sc, device="cuda:0")
    rc, (rgb, depth, alpha) = _noalloc(ds, D.dgs_default_options())
    assert rc == D.DGS_OK
    v = 1
    e, c = sc.views[v]
    ref = O.render_view(sc, e, c)
    H, W = ref.depth.shape
    sl = ds.view_slice(v)
    bad, rep = compare_view(rgb[sl].reshape(H, W, 3), depth[sl].reshape(H, W), ref, alpha[sl].reshape(H, W))
    assert bad == 0, rep


def test_noalloc_rejects_batches_beyond_its_scratch():
    from paper_2507_21981_gb300.render import DeviceScene
    # tables of 128 views x 33,750 chunks do not fit: rejected while the tables are sized
    sc = S.config2(seed=6, n_envs=64, n_bg=1_000_000, n_obj=20_000, width=640, height=480)
    ds = DeviceScene(sc, device="cuda:0")
    rc, _ = _noalloc(ds, D.dgs_default_options())
    assert rc == D.DGS_ERR_CAPACITY


def test_noalloc_rejects_records_beyond_its_scratch_then_renders_again():
    """One view of 1.2M Gaussians that are all in front of the camera: the tables fit, the
    projected records (80 B each) do not, so the call stops after its count pass with
    DGS_ERR_CAPACITY; an ordinary batch right after it still equals dgs_render bit for bit."""
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    big = DeviceScene(S.config1(seed=2, n_bg=1_200_000, n_obj=1_000, res=128, f=110.0), device="cuda:0")
    rc, _ = _noalloc(big, D.dgs_default_options())
    assert rc == D.DGS_ERR_CAPACITY
    da = DeviceScene(_scene_a(), device="cuda:0")
    r = Renderer(mode="batched")
    ref = _render(r, da)
    rc, got = _noalloc(da, r.options)
    assert rc == D.DGS_OK
    _same(got, ref, "after the rejected batch")
    r.close()


def test_noalloc_rejects_the_cameras_render_rejects():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    ds = DeviceScene(_scene_b(), device="cuda:0")
    r = Renderer(mode="batched")
    for field, index, value in (("cam_from_world", 3, float("nan")), ("fx", None, float("inf")),
                                ("cy", None, float("nan")), ("cam_from_world", 11, float("inf"))):
        cams = type(ds.cams).from_buffer_copy(ds.cams)
        if index is None:
            setattr(cams[0], field, value)
        else:
            getattr(cams[0], field)[index] = value
        rc, _ = _noalloc(ds, D.dgs_default_options(), cams=cams)
        assert rc == D.DGS_ERR_INVALID_ARG, (field, index, rc)
        n = ds.n_pixels
        rc2 = D.dgs_render(r.ctx, ds.nodes, ds.n_nodes, ds.env_node_ids, ds.n_envs, ds.max_nodes, ds.node_poses,
                           cams, ds.cams_per_env, ds.max_cams, torch.empty((n, 3), device=ds.device),
                           torch.empty((n,), device=ds.device), None, None, torch.cuda.current_stream().cuda_stream)
        assert rc2 == D.DGS_ERR_INVALID_ARG, (field, index, rc2)
    r.close()
