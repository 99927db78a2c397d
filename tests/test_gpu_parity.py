"""GPU (libdgs through the C ABI) vs the FP64 oracle, pixel by pixel, on seeded scenes."""
import numpy as np
import pytest

import oracle as O
from paper_2507_21981_gb300 import scenes as S
from tests.parity import compare_view

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OPTS = O.OracleOptions()


def _render(sc, mode="batched", dtype="f32", spatial_order=False, **kw):
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    ds = DeviceScene(sc, device="cuda:0", dtype=dtype, spatial_order=spatial_order)
    r = Renderer(mode=mode, **kw)
    rgb, depth, alpha = r.render(ds)
    torch.cuda.synchronize()
    out = rgb.cpu().numpy(), depth.cpu().numpy(), alpha.cpu().numpy()
    stats, launches = r.stats(), r.launches()
    r.close()
    return ds, out, stats, launches


def _check_views(sc, ds, out, views, opts=OPTS, packed=None):
    rgb, depth, alpha = out
    reports = []
    for v in views:
        e, c = sc.views[v]
        ref = O.render_view(sc, e, c, opts, packed)
        H, W = ref.depth.shape
        sl = ds.view_slice(v)
        bad, rep = compare_view(rgb[sl].reshape(H, W, 3), depth[sl].reshape(H, W), ref, alpha[sl].reshape(H, W))
        rep["view"] = v
        reports.append(rep)
        assert bad == 0, rep
        # the plain relative depth bound, without the coverage term, on every unambiguous pixel
        assert rep["frac_depth_plain_over_1e4_unambiguous"] == 0.0, rep
    return reports


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_config1_every_pixel(mode):
    sc = S.config1(seed=1)
    ds, out, st, launches = _render(sc, mode)
    assert launches > 0 and st["n_visible"] > 0
    reps = _check_views(sc, ds, out, [0])
    assert reps[0]["ambiguous"] / reps[0]["pixels"] < 1e-2


@pytest.mark.parametrize("seed", [2, 3])
def test_config1_more_seeds_and_background(seed):
    sc = S.config1(seed=seed)
    ds, out, _, _ = _render(sc, "batched", bg=(0.2, 0.4, 0.6))
    _check_views(sc, ds, out, [0], O.OracleOptions(bg=(0.2, 0.4, 0.6)))


def test_config2_reduced_all_views():
    # the config-2 law at reduced size: 4 envs x 2 cameras 160x120, 60k room + 4 x 2k objects
    sc = S.config2(seed=1, n_envs=4, n_bg=60_000, n_obj=2_000, width=160, height=120, f=125.0)
    ds, out, st, _ = _render(sc, "batched")
    assert st["n_views"] == 8
    _check_views(sc, ds, out, range(8))


def test_batched_equals_plain_bitwise():
    sc = S.config2(seed=2, n_envs=3, n_bg=40_000, n_obj=1_500, width=160, height=120, f=125.0)
    _, a, _, _ = _render(sc, "batched")
    _, b, _, _ = _render(sc, "plain")
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("test_fault", [0, 4])
def test_group_of_more_than_256_views_equals_plain_bitwise(test_fault):
    """150 envs x 2 cameras of 64x48 in one view group: the view key of the depth sort has 9
    bits and takes two passes (5 + 4 bits), carried in the instance numbers' high bits or, with
    test_fault 4, gathered from the view array.  The batched render must equal the plain
    per-view render (one view per group, no view passes) bit for bit, and match the oracle."""
    sc = S.config2(seed=6, n_envs=150, n_bg=20_000, n_obj=500, width=64, height=48, f=50.0)
    ds, a, st, _ = _render(sc, "batched", views_per_group=300, test_fault=test_fault)
    assert st["n_views"] == 300 and st["n_groups"] == 1 and st["n_pairs"] > 0
    _, b, _, _ = _render(sc, "plain")
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    _check_views(sc, ds, a, [0, 157, 299])


@pytest.mark.parametrize("spatial_order", [False, True])
def test_config3_reduced_ragged_views(spatial_order):
    sc = S.config3(seed=1, n_envs=6, n_bg=30_000, n_assets=8, asset_lo=500, asset_hi=4_000, max_nodes=4,
                   resolutions=((80, 60), (160, 120), (200, 110)))
    ds, out, st, _ = _render(sc, "batched", spatial_order=spatial_order)
    _check_views(ds.scene, ds, out, range(sc.n_views))


def test_ragged_tiles_and_tile_shapes():
    sc = S.config1(seed=4, res=100, f=86.0)     # 100x100: partial tiles at the right/bottom
    for tile in [(16, 16), (32, 8), (8, 32), (16, 8), (8, 8), (64, 4), (32, 4), (16, 4)]:
        ds, out, _, _ = _render(sc, "batched", tile=tile)
        _check_views(sc, ds, out, [0])


def test_views_per_group_split_matches_single_group():
    sc = S.config2(seed=3, n_envs=3, n_bg=20_000, n_obj=1_000, width=96, height=64, f=75.0)
    _, a, st1, _ = _render(sc, "batched")
    _, b, st2, _ = _render(sc, "batched", views_per_group=2)
    assert st1["n_groups"] == 1 and st2["n_groups"] == 3
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_empty_nodes_and_env_without_cameras():
    sc = S.config2(seed=4, n_envs=3, n_bg=5_000, n_obj=500, width=64, height=48, f=50.0)
    sc.cams_per_env[1] = 0                       # an env with no camera
    sc.nodes[2] = sc.nodes[2].subset(slice(0, 0))  # an empty node
    ds, out, st, _ = _render(sc, "batched")
    assert st["n_views"] == 4
    _check_views(sc, ds, out, range(4))


def test_all_transparent_scene_gives_background():
    sc = S.config1(seed=5)
    for nd in sc.nodes:
        nd.opacity_logit[:] = -30.0
    ds, out, st, _ = _render(sc, "batched", bg=(0.1, 0.2, 0.3))
    rgb, depth, alpha = out
    assert np.allclose(rgb, [0.1, 0.2, 0.3], atol=1e-7) and np.all(depth == 0) and np.all(alpha == 0)


@pytest.mark.parametrize("mode", ["batched", "graph"])
def test_config2_full_size_sampled_views(mode):
    """Full workload of the benchmark (64 envs x 2 cams 640x480, 1.08M Gaussians, nodes in
    Z-order as the benchmark stores them); the oracle checks two seeded sampled views pixel by
    pixel of the permuted scene."""
    sc = S.config2(seed=1)
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    ds = DeviceScene(sc, device="cuda:0", spatial_order=True)
    r = Renderer(mode=mode)
    for _ in range(2 if mode == "graph" else 1):     # graph: the second call replays
        out = [t.cpu().numpy() for t in r.render(ds)]
    st = r.stats()
    r.close()
    assert st["n_views"] == 128 and st["n_groups"] >= 1 and st["path"] == (1 if mode == "graph" else 0)
    views = sorted(int(v) for v in np.random.default_rng(7).choice(sc.n_views, 2, replace=False))
    _check_views(ds.scene, ds, out, views, packed=O.oracle._Packed(ds.scene))


def test_spatial_order_reduced_all_views_and_nearly_equal_image():
    """Z-ordered storage: every view against the oracle of the permuted scene.  Against the
    original order the image changes only where two Gaussians reaching a pixel share a depth
    key bit for bit (their id order follows the permutation): a few pixels in 1e5."""
    sc = S.config2(seed=1, n_envs=4, n_bg=60_000, n_obj=2_000, width=160, height=120, f=125.0)
    ds, out, st, _ = _render(sc, "batched", spatial_order=True)
    _check_views(ds.scene, ds, out, range(8))
    _, ref, st0, _ = _render(sc, "batched")
    assert st["n_visible"] == st0["n_visible"] and st["n_pairs"] == st0["n_pairs"]
    differ = np.any(out[0] != ref[0], axis=1) | (out[1] != ref[1])
    assert differ.mean() < 1e-3, int(differ.sum())


def _cluster(rng, n, centre, spread, log_sigma, opacity_logit):
    mean = (np.asarray(centre) + rng.uniform(-spread, spread, (n, 3))).astype(np.float32)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    sh = rng.uniform(-1.0, 1.0, (n, 1, 3)).astype(np.float32)
    return S.GaussianNode(mean, np.full((n, 3), log_sigma, np.float32), q,
                          np.full(n, opacity_logit, np.float32), sh, 0, "cluster")


def test_chunk_cull_keeps_gaussians_that_bleed_into_the_image():
    """Camera at (0,0,-5) looking along +z, 128x128, f = 110: at depth 5 the image edges lie at
    |x|, |y| = 2.909.  Four 32-Gaussian clusters sit just outside the four edges (centres about
    2 px beyond them, sigma 2.2 px) and reach back into the image; one straddles the near plane;
    one lies far outside (its chunk is culled); a cloud fills the middle.  The per-chunk cull
    must keep every Gaussian whose ellipse reaches a pixel."""
    rng = np.random.default_rng(0)
    e = 5.0 * 64.0 / 110.0
    parts = [_cluster(rng, 32, c, 0.04, np.log(0.1), 3.0)
             for c in [(-e - 0.1, 0, 0), (e + 0.1, 0.5, 0), (0.4, -e - 0.1, 0), (-0.3, e + 0.1, 0)]]
    parts.append(_cluster(rng, 32, (0.0005, 0.0003, -4.99), 0.004, np.log(0.0005), -1.0))
    parts.append(_cluster(rng, 32, (-e - 3.0, 0, 0), 0.04, np.log(0.1), 3.0))
    parts.append(_cluster(rng, 256, (0, 0, 0), 1.5, np.log(0.05), 0.0))
    node = S.GaussianNode(*(np.concatenate([getattr(p, f) for p in parts]) for f in
                            ("mean", "log_scale", "quat", "opacity_logit", "sh")), 0, "edges")
    I = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    cam = np.concatenate([np.eye(3), np.array([[0.0], [0.0], [5.0]])], axis=1)
    sc = S.scene_from_lists("edges", [node], [[0]], [[I]], [[(110.0, 110.0, 64.0, 64.0, 128, 128, cam)]])
    for mode in ("batched", "plain"):
        ds, out, _, _ = _render(sc, mode, spatial_order=True)
        _check_views(ds.scene, ds, out, [0])
    ref = O.render_view(sc, 0, 0, OPTS)
    a = ref.alpha                                      # the border coverage comes from the edge clusters
    assert a[:, 0].max() > 0.2 and a[:, -1].max() > 0.2 and a[0, :].max() > 0.2 and a[-1, :].max() > 0.2


def test_config4_full_view():
    sc = S.config4(seed=1)
    ds, out, st, _ = _render(sc, "batched")
    _check_views(sc, ds, out, [0])
