"""Failure detection on the GPU without a GPU fault: a bounded device-side wait that runs out,
and the host-side checker of the binning invariants.

The onesweep sort's decoupled look-back waits, with a wall-clock limit, for the status of the
partitions before it.  dgs_options.test_fault = 1 makes one partition of the depth sort's first
pass publish nothing, so the waits behind it run out after spin_limit_us: the call must return
DGS_ERR_TIMEOUT (the kernels that would read the invalid sort skip their work), and the next
call on the same context, with the fault cleared, must render the correct image.
dgs_options.check_binning reads each view group's tile lists back and checks them on the host;
test_fault = 2 corrupts the host copy before the check, which must report it.
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_21981_gb300 import dgs as D
from paper_2507_21981_gb300 import scenes as S
from tests.parity import compare_view

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _check_oracle(sc, ds, out, v=0):
    rgb, depth, alpha = (t.cpu().numpy() for t in out)
    e, c = sc.views[v]
    ref = O.render_view(sc, e, c)
    H, W = ref.depth.shape
    sl = ds.view_slice(v)
    bad, rep = compare_view(rgb[sl].reshape(H, W, 3), depth[sl].reshape(H, W), ref, alpha[sl].reshape(H, W))
    assert bad == 0, rep


def test_sort_wait_runs_out_then_the_context_renders_again():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config1(seed=1)                      # about 10k visible instances: 3 sort partitions
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer(mode="batched", spin_limit_us=2000, test_fault=1)
    with pytest.raises(D.DgsError) as ei:
        r.render(ds)
    assert ei.value.code == D.DGS_ERR_TIMEOUT
    assert "timed out" in D.dgs_last_error(r.ctx)
    r.set_options(test_fault=0)
    out = r.render(ds)
    torch.cuda.synchronize()
    _check_oracle(sc, ds, out)
    r.close()


def test_default_spin_limit_does_not_fire_on_a_full_batch():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config2(seed=3, n_envs=8, n_bg=200_000, n_obj=5_000, width=320, height=240, f=250.0)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer(mode="batched", spin_limit_us=200_000)
    r.render(ds)
    torch.cuda.synchronize()
    assert r.stats()["n_pairs"] > 0
    r.close()


@pytest.mark.parametrize("make", [
    lambda: S.config1(seed=2),
    lambda: S.config2(seed=4, n_envs=3, n_bg=30_000, n_obj=1_000, width=160, height=120, f=125.0),
    lambda: S.config3(seed=2, n_envs=5, n_bg=20_000, n_assets=6, asset_lo=500, asset_hi=3_000, max_nodes=3,
                      resolutions=((80, 60), (160, 120), (200, 110))),
])
@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_binning_invariants_hold(make, tile):
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = make()
    ds = DeviceScene(sc, device="cuda:0", spatial_order=True)
    r = Renderer(mode="batched", tile=tile, check_binning=1, views_per_group=2)
    out = r.render(ds)
    torch.cuda.synchronize()
    assert r.stats()["n_pairs"] > 0
    _check_oracle(ds.scene, ds, out)
    r.close()


def test_binning_checker_reports_a_corrupted_list():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config1(seed=3)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer(mode="batched", check_binning=1, test_fault=2)
    with pytest.raises(D.DgsError) as ei:
        r.render(ds)
    assert ei.value.code == D.DGS_ERR_CUDA and "binning invariant violated" in str(ei.value)
    r.set_options(test_fault=0)
    out = r.render(ds)
    torch.cuda.synchronize()
    _check_oracle(sc, ds, out)
    r.close()


@pytest.mark.parametrize("mode", ["batched", "graph"])
@pytest.mark.parametrize("bad", ["nan", "scaled"])
def test_corrupted_node_pose_is_reported_then_the_context_renders_again(mode, bad):
    """Fault injection on the host: one node pose of the batch is made non-finite or non-rigid
    (rotation scaled by 2) in the caller's pose array.  The device-side pose check must end the
    render and the backward with DGS_ERR_INVALID_ARG, and the same context must render the
    restored poses exactly as before."""
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config2(seed=4, n_envs=3, n_bg=30_000, n_obj=1_000, width=160, height=120, f=125.0)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer(mode=mode)
    ref = [t.cpu().numpy() for t in r.render(ds)]
    if mode == "graph":
        ref = [t.cpu().numpy() for t in r.render(ds)]      # a replay of the captured sequence
    good = ds.node_poses.clone()
    if bad == "nan":
        ds.node_poses[1, 1, 3] = float("nan")
    else:
        ds.node_poses[1, 1, :] = ds.node_poses[1, 1, :] * torch.tensor([2, 2, 2, 1] * 3, dtype=torch.float32,
                                                                         device=ds.device)
    with pytest.raises(D.DgsError) as ei:
        r.render(ds)
    assert ei.value.code == D.DGS_ERR_INVALID_ARG and "not finite or not rigid" in str(ei.value)
    rgb, depth = (torch.as_tensor(x, device=ds.device) for x in ref[:2])
    with pytest.raises(D.DgsError) as ei:
        r.backward(ds, rgb, depth, torch.ones_like(rgb), torch.ones_like(depth))
    assert ei.value.code == D.DGS_ERR_INVALID_ARG
    ds.node_poses.copy_(good)
    out = [t.cpu().numpy() for t in r.render(ds)]
    torch.cuda.synchronize()
    for a, b in zip(ref, out):
        assert np.array_equal(a, b)
    r.close()


@pytest.mark.parametrize("mode", ["batched", "graph"])
def test_gathered_view_key_renders_what_the_packed_one_does(mode):
    """The depth sort's view key rides in the instance numbers' high bits where both fit in 32
    bits, else it is gathered from a per-instance view array (large view groups).  test_fault = 4
    forces the gathered form on a small batch: the tile lists (checked on the host in the eager
    render) and the images must equal the packed form's bit for bit, and the image the oracle's."""
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config2(seed=5, n_envs=6, n_bg=30_000, n_obj=1_000, width=160, height=120, f=125.0)
    ds = DeviceScene(sc, device="cuda:0", spatial_order=True)
    outs = []
    for tf in (0, 4):
        kw = {"check_binning": 1} if mode == "batched" else {}
        r = Renderer(mode=mode, test_fault=tf, **kw)
        out = r.render(ds)
        if mode == "graph":
            out = r.render(ds)                  # a replay of the captured sequence
        torch.cuda.synchronize()
        if mode == "batched":
            assert r.stats()["n_groups"] == 1 and r.stats()["n_pairs"] > 0
        outs.append([t.cpu().numpy() for t in out])
        r.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    _check_oracle(ds.scene, ds, [torch.as_tensor(x) for x in outs[1]], v=3)
