"""dgs_render_noalloc, the render for callers that cannot allocate GPU memory.

Such a caller (a program whose device memory belongs to another framework's caching
allocator, a control loop that cannot afford the synchronisation of cudaMalloc/cudaFree in a
step, code certified to allocate nothing after start-up) passes its inputs and outputs and
gets the same images as dgs_render, while the library works inside its fixed 64 MiB array.
This file is collected last on purpose: the test must also pass after every other test.
"""
import numpy as np
import pytest

from paper_2507_21981_gb300 import dgs as D
from paper_2507_21981_gb300 import scenes as S
from tests.parity import D_FLOOR, TOL_DREL, TOL_RGB

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(ds, opts, stream, out=None):
    n = ds.n_pixels
    if out is None:
        out = (torch.empty((n, 3), device=ds.device), torch.empty((n,), device=ds.device),
               torch.empty((n,), device=ds.device))
    for t in out:
        t.fill_(-1.0)
    rgb, depth, alpha = out
    rc = D.dgs_render_noalloc(opts, ds.nodes, ds.n_nodes, ds.env_node_ids, ds.n_envs, ds.max_nodes, ds.node_poses,
                              ds.cams, ds.cams_per_env, ds.max_cams, rgb, depth, alpha, None, stream.cuda_stream)
    return rc, rgb, depth, alpha


def test_noalloc_matches_render_twice_in_a_row():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config2(seed=5, n_envs=3, n_bg=40_000, n_obj=1_500, width=160, height=120, f=125.0)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer(mode="batched")
    ref_rgb, ref_d, ref_a = (t.cpu().numpy() for t in r.render(ds))
    stream = torch.cuda.current_stream()
    n = ds.n_pixels
    out = (torch.empty((n, 3), device=ds.device), torch.empty((n,), device=ds.device),
           torch.empty((n,), device=ds.device))
    moved = []
    for call in range(2):
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc, rgb, depth, alpha = _noalloc(ds, r.options, stream, out)
        torch.cuda.synchronize()
        moved.append(free_before - torch.cuda.mem_get_info()[0])
        assert rc == D.DGS_OK, D.STATUS_NAMES.get(rc, rc)
        g_rgb, g_d, g_a = rgb.cpu().numpy(), depth.cpu().numpy(), alpha.cpu().numpy()
        e_a = np.abs(g_a - ref_a)
        assert np.abs(g_rgb - ref_rgb).max() <= TOL_RGB and e_a.max() <= TOL_RGB
        surface = np.where(ref_a > 1e-12, np.abs(ref_d) / np.maximum(ref_a, 1e-12), 0.0)
        assert np.all(np.abs(g_d - ref_d) <= TOL_DREL * np.maximum(np.abs(ref_d), D_FLOOR) + e_a * surface), call
    # no device memory taken by the library during the second call (the first may still load code)
    assert moved[1] == 0, moved
    r.close()


def test_noalloc_rejects_batches_beyond_its_scratch():
    from paper_2507_21981_gb300.render import DeviceScene
    sc = S.config2(seed=6, n_envs=64, n_bg=1_000_000, n_obj=20_000, width=640, height=480)
    ds = DeviceScene(sc, device="cuda:0")
    rc, *_ = _noalloc(ds, D.dgs_default_options(), torch.cuda.current_stream())
    assert rc == D.DGS_ERR_CAPACITY
