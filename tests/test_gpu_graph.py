"""Graph replay (DGS_MODE_GRAPH) and the tile-shape autotuner, through the C ABI.

The replayed graph runs the same kernels on the same inputs in the same order as the eager
batched sequence with one view group, so its images must equal the eager ones bit for bit;
the eager sequence is itself checked against the FP64 oracle (test_gpu_parity.py), and one
ragged batch is checked against the oracle here directly.  Every tile shape yields the same
per-pixel list (all Gaussians whose ellipse holds the pixel centre, in (z32, id) order), so
images are also bit-identical across tile shapes.
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_21981_gb300 import scenes as S
from tests.parity import compare_view

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ragged():
    return S.config3(seed=5, n_envs=7, n_bg=30_000, n_assets=8, asset_lo=500, asset_hi=4_000, max_nodes=4,
                     resolutions=((80, 60), (160, 120), (200, 110)))


def _eager(sc, ds_poses=None, **kw):
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    ds = DeviceScene(sc, device="cuda:0")
    if ds_poses is not None:
        ds.set_poses(ds_poses)
    r = Renderer(mode="batched", **kw)
    out = [t.cpu().numpy() for t in r.render(ds)]
    r.close()
    return out


def _host(out):
    return [t.cpu().numpy() for t in out]


def _equal(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_graph_replay_equals_eager_bitwise_and_follows_new_poses():
    from paper_2507_21981_gb300 import dgs as D
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = _ragged()
    ref = _eager(sc)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer(mode="graph")
    _equal(_host(r.render(ds)), ref)
    assert r.stats()["path"] == D.DGS_PATH_CAPTURED and r.stats()["graph_captures"] == 1
    for _ in range(2):
        _equal(_host(r.render(ds)), ref)
        st = r.stats()
        assert st["path"] == D.DGS_PATH_GRAPH and st["graph_captures"] == 1
        assert r.launches() > 8
    # new object poses, same structure: the replay reads them from the pose buffer
    rng = np.random.default_rng(11)
    poses = sc.node_poses.copy()
    for e in range(sc.n_envs):
        for j in range(1, poses.shape[1]):
            if sc.env_node_ids[e, j] >= 0:
                poses[e, j] = S.workspace_pose(rng)
    ds.set_poses(poses)
    got = _host(r.render(ds))
    assert r.stats()["path"] == D.DGS_PATH_GRAPH
    moved = S.Scene(sc.name, sc.nodes, sc.env_node_ids, poses, sc.cams_per_env, sc.cam_intr, sc.cam_res,
                    sc.cam_pose, sc.meta)
    _equal(got, _eager(moved))
    # the replay against the oracle on every ragged view of the moved batch
    rgb, depth, alpha = got
    pk = O.oracle._Packed(moved)
    for v, (e, c) in enumerate(moved.views):
        ref_v = O.render_view(moved, e, c, O.OracleOptions(), pk)
        H, W = ref_v.depth.shape
        sl = ds.view_slice(v)
        bad, rep = compare_view(rgb[sl].reshape(H, W, 3), depth[sl].reshape(H, W), ref_v, alpha[sl].reshape(H, W))
        assert bad == 0, rep
    r.close()


def test_graph_overflow_renders_eagerly_and_recaptures():
    """First call with the object behind the camera (few pairs), then in front of it: the
    replay overflows its capacity, the call re-renders eagerly, and the next call replays the
    recaptured graph."""
    from paper_2507_21981_gb300 import dgs as D
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config1(seed=7, n_bg=1_000, n_obj=20_000)
    far = sc.node_poses.copy()
    far[0, 1, :, 3] = [0.0, 0.0, -100.0]         # object node 95 m behind the camera: culled
    near = sc.node_poses.copy()
    ds = DeviceScene(sc, device="cuda:0")
    ds.set_poses(far)
    r = Renderer(mode="graph")
    r.render(ds)
    st0 = r.stats()
    assert st0["path"] == D.DGS_PATH_CAPTURED
    ds.set_poses(near)
    got = _host(r.render(ds))
    st1 = r.stats()
    assert st1["path"] == D.DGS_PATH_REGROWN and st1["graph_captures"] == 2
    assert st1["n_pairs"] > 1.25 * st0["n_pairs"] + 4096
    _equal(got, _eager(sc))
    got2 = _host(r.render(ds))
    assert r.stats()["path"] == D.DGS_PATH_GRAPH
    _equal(got2, got)
    # back to the small batch: replays within capacity
    ds.set_poses(far)
    _host(r.render(ds))
    assert r.stats()["path"] == D.DGS_PATH_GRAPH
    r.close()


def test_graph_recaptures_for_new_output_buffers():
    from paper_2507_21981_gb300 import dgs as D
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config1(seed=8)
    ref = _eager(sc)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer(mode="graph")
    r.render(ds)
    outs = [torch.empty((ds.n_pixels, 3), device="cuda:0"), torch.empty(ds.n_pixels, device="cuda:0"), None]
    got = r.render(ds, out=outs)
    assert r.stats()["path"] == D.DGS_PATH_CAPTURED and r.stats()["graph_captures"] == 2
    _equal(_host(got[:2]), ref[:2])
    r.close()


def test_tile_shapes_give_identical_images():
    sc = _ragged()
    ref = _eager(sc)
    for tile in [(32, 8), (8, 32), (16, 8), (8, 8)]:
        _equal(_eager(sc, tile=tile), ref)
    _equal(_eager(sc, exact_tile_test=0), ref)


@pytest.mark.parametrize("mode", ["batched", "graph"])
def test_autotune_picks_a_candidate_and_renders_with_it(mode):
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = _ragged()
    ref = _eager(sc)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer(mode=mode)
    best, times, out = r.autotune(ds, reps=2)
    assert set(times) == {(16, 16), (32, 8), (8, 32), (16, 8), (8, 8)}
    assert all(t > 0 for t in times.values()) and times[best] == min(times.values())
    _equal(_host(out), ref)
    _equal(_host(r.render(ds)), ref)
    best2, times2, _ = r.autotune(ds, candidates=[(8, 8), (16, 16)], reps=1)
    assert set(times2) == {(8, 8), (16, 16)} and best2 in times2
    r.close()


def test_config3_full_size_graph_sampled_views():
    """The uneven workload at full size (256 envs, 1-12 assets of 5k-200k Gaussians, 1-3
    cameras at three resolutions, 504 views, Z-ordered nodes) rendered as a graph replay after
    dgs_autotune; one sampled view of each resolution against the oracle."""
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config3(seed=1)
    ds = DeviceScene(sc, device="cuda:0", spatial_order=True)
    r = Renderer(mode="graph")
    r.autotune(ds, reps=1)
    rgb, depth, alpha = [t.cpu().numpy() for t in r.render(ds)]
    assert r.stats()["path"] == 1
    r.close()
    rng = np.random.default_rng(5)
    picked = {}
    for v in rng.permutation(sc.n_views):
        w, h = (int(x) for x in sc.view_res(int(v)))
        picked.setdefault((w, h), int(v))
    pk = O.oracle._Packed(ds.scene)
    for (w, h), v in sorted(picked.items()):
        e, c = sc.views[v]
        ref = O.render_view(ds.scene, e, c, O.OracleOptions(), pk)
        sl = ds.view_slice(v)
        bad, rep = compare_view(rgb[sl].reshape(h, w, 3), depth[sl].reshape(h, w), ref, alpha[sl].reshape(h, w))
        assert bad == 0, (w, h, rep)
    assert len(picked) == 3


def test_autotune_cache_reuses_the_shape_of_a_known_class(tmp_path):
    from paper_2507_21981_gb300.render import DeviceScene, Renderer, TuneCache
    cache = TuneCache(str(tmp_path / "tune.json"))
    sc = S.config1(seed=2)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer(mode="batched")
    best, times, _ = r.autotune(ds, candidates=[(16, 16), (8, 8), (32, 8)], reps=1, cache=cache)
    assert not r.tune_cached and best in times
    # another scene of the same class (same resolution, Gaussians per view within a factor of 2)
    ds2 = DeviceScene(S.config1(seed=3), device="cuda:0")
    r2 = Renderer(mode="batched")
    best2, times2, out = r2.autotune(ds2, reps=1, cache=cache)
    assert r2.tune_cached and best2 == best and times2 == times
    assert (r2.options.tile_w, r2.options.tile_h) == best
    rgb, depth, alpha = (t.cpu().numpy() for t in out)
    torch.cuda.synchronize()
    r3 = Renderer(mode="batched", tile=best)
    ref = [t.cpu().numpy() for t in r3.render(ds2)]
    for a, b in zip((rgb, depth, alpha), ref):
        assert np.array_equal(a, b)
    for x in (r, r2, r3):
        x.close()
