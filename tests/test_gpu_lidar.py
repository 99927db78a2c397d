"""LiDAR Gaussian ray tracing (dgs_lidar_build / dgs_lidar_trace) against the FP64 oracle.

Every ray's D (= sum w t*) and A (= 1 - T) must lie within twice the tolerance the oracle
derives for that ray from an FP32 error model (oracle/lidar.cpp: continuous errors plus the
effect of every decision FP32 may take the other way), plus 1e-6 absolute.  Cases: a dense
cube of Gaussians, ragged multi-env scenes with posed nodes in storage order and in Z-order,
BF16 storage (oracle fed the same rounded attributes), edge cases (nodes of 0, 1, 8 and 9
Gaussians, an env without nodes, axis-parallel rays, a sensor inside a Gaussian, an empty range
window), a rebuild after the attributes change, and the full benchmark batch (64 sensors x
32 x 1024 rays through the 1.08M-Gaussian scene) on sampled rays.
"""
import numpy as np
import pytest

from oracle import lidar as OL
from oracle import oracle as OO
from paper_2507_21981_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _check(d, a, ref, what=""):
    d = np.asarray(d, np.float64)
    a = np.asarray(a, np.float64)
    ea, ed = np.abs(a - ref.a), np.abs(d - ref.d)
    ta, td = 2 * ref.tol_a + 1e-6, 2 * ref.tol_d + 1e-6 * (1 + np.abs(ref.d))
    bad = (ea > ta) | (ed > td)
    rep = dict(what=what, rays=int(a.size), bad=int(bad.sum()), hit=int((ref.a > 0.5).sum()),
               max_err_a=float(ea.max()), max_err_d=float(ed.max()),
               max_ratio_a=float((ea / ta).max()), max_ratio_d=float((ed / td).max()))
    if bad.any():
        i = np.unravel_index(np.argmax(np.maximum(ea / ta, ed / td)), a.shape)
        rep["worst"] = dict(index=[int(x) for x in i], gpu=[float(d[i]), float(a[i])], oracle=[float(ref.d[i]), float(ref.a[i])],
                            tol=[float(ref.tol_d[i]), float(ref.tol_a[i])], n_comp=int(ref.n_comp[i]),
                            n_amb=int(ref.n_amb[i]))
    assert not bad.any(), rep
    return rep


def _trace(ds, se, sp, dirs, r_min=0.05, r_max=30.0, build=True, r=None):
    from paper_2507_21981_gb300.render import Renderer
    own = r is None
    r = r or Renderer()
    if build:
        r.lidar_build(ds)
    d_dirs = torch.as_tensor(np.ascontiguousarray(dirs, np.float32)).cuda()
    D, A = r.lidar_trace(ds, se, sp, d_dirs, r_min, r_max)
    out = D.cpu().numpy(), A.cpu().numpy()
    if own:
        r.close()
    return out


def _oracle(sc, se, sp, dirs, r_min=0.05, r_max=30.0, packed=None):
    return OL.trace(sc, se, sp, np.asarray(dirs, np.float32), OL.LidarOptions(r_min=r_min, r_max=r_max), packed=packed)


@pytest.mark.parametrize("zorder", [False, True])
def test_dense_cube_matches_oracle(zorder):
    from paper_2507_21981_gb300.render import DeviceScene
    sc = S.config1(seed=3)
    ds = DeviceScene(sc, device="cuda:0", spatial_order=zorder)
    se, sp = S.lidar_sensors(3, sc.n_envs)
    dirs = S.lidar_pattern(16, 256)
    d, a = _trace(ds, se, sp, dirs)
    rep = _check(d, a, _oracle(ds.scene, se, sp, dirs), f"cube zorder={zorder}")
    assert rep["hit"] > 1000


def _ragged():
    return S.config3(seed=5, n_envs=7, n_bg=30_000, n_assets=8, asset_lo=500, asset_hi=4_000, max_nodes=4,
                     resolutions=((80, 60), (160, 120), (200, 110)))


@pytest.mark.parametrize("zorder", [False, True])
def test_ragged_posed_nodes_match_oracle(zorder):
    from paper_2507_21981_gb300.render import DeviceScene
    sc = _ragged()
    ds = DeviceScene(sc, device="cuda:0", spatial_order=zorder)
    se, sp = S.lidar_sensors(5, sc.n_envs)
    dirs = S.lidar_pattern(12, 192)
    d, a = _trace(ds, se, sp, dirs)
    _check(d, a, _oracle(ds.scene, se, sp, dirs), f"ragged zorder={zorder}")


def test_bf16_storage_matches_oracle_on_rounded_attributes():
    from paper_2507_21981_gb300.render import DeviceScene
    sc = _ragged()
    ds = DeviceScene(sc, device="cuda:0", dtype="bf16", spatial_order=True)
    rd = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(torch.bfloat16).float().numpy()
    rs = S.Scene(ds.scene.name, [S.GaussianNode(nd.mean, rd(nd.log_scale), rd(nd.quat), nd.opacity_logit, nd.sh,
                                                nd.sh_degree, nd.name) for nd in ds.scene.nodes],
                 sc.env_node_ids, sc.node_poses, sc.cams_per_env, sc.cam_intr, sc.cam_res, sc.cam_pose, sc.meta)
    se, sp = S.lidar_sensors(6, sc.n_envs)
    dirs = S.lidar_pattern(8, 128)
    d, a = _trace(ds, se, sp, dirs)
    _check(d, a, _oracle(rs, se, sp, dirs), "bf16")


def _tiny(rng, n, centre):
    from scipy.spatial.transform import Rotation
    q = Rotation.random(max(n, 1), random_state=int(rng.integers(1 << 30))).as_quat()[:n]
    f = np.float32
    return S.GaussianNode((centre + rng.uniform(-0.3, 0.3, (n, 3))).astype(f), rng.uniform(-3.0, -1.5, (n, 3)).astype(f),
                          np.concatenate([q[:, 3:], q[:, :3]], axis=1).astype(f), rng.normal(1.0, 1.0, n).astype(f),
                          np.zeros((n, 1, 3), f), 0, "tiny")


def test_edge_cases():
    """Nodes of 0, 1, 8 and 9 Gaussians (empty tree, a root that is a leaf, one full leaf, two
    leaves), an env holding no node, axis-parallel rays (infinite slab reciprocals), a sensor
    inside a Gaussian, and an empty range window."""
    from paper_2507_21981_gb300.render import DeviceScene
    rng = np.random.default_rng(7)
    nodes = [_tiny(rng, 0, np.zeros(3)), _tiny(rng, 1, np.array([1.0, 0, 0])), _tiny(rng, 8, np.array([1.5, 0.2, 0])),
             _tiny(rng, 9, np.array([0.0, 1.2, 0.1]))]
    inside = _tiny(rng, 1, np.zeros(3))
    inside.mean[:] = [0.01, 0.0, 0.0]
    inside.log_scale[:] = [-1.0, -1.0, -1.0]
    nodes.append(inside)
    P = S.random_pose(rng, 0.05)
    env_nodes = [[0, 1, 2, 3], [], [4, 2]]
    env_poses = [[np.eye(3, 4), np.eye(3, 4), P, np.eye(3, 4)], [], [np.eye(3, 4), np.eye(3, 4)]]
    cams = [[(50.0, 50.0, 16.0, 16.0, 32, 32, np.eye(3, 4))]] * 3
    sc = S.scene_from_lists("edge", nodes, env_nodes, env_poses, cams)
    ds = DeviceScene(sc, device="cuda:0")
    dirs = np.concatenate([S.lidar_pattern(8, 64, -40, 40),
                           np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [-1, 0, 0], [0, -1, 0], [0, 0, -1]], np.float32)])
    se = np.array([0, 1, 2, 0], np.int32)
    sp = np.repeat(np.eye(3, 4, dtype=np.float32)[None], 4, axis=0)
    sp[3, :, 3] = [0.2, 0.1, 0.0]
    from paper_2507_21981_gb300.render import Renderer
    r = Renderer()
    d, a = _trace(ds, se, sp, dirs, r=r)
    ref = _oracle(sc, se, sp, dirs)
    _check(d, a, ref, "edge")
    assert np.all(a[1] == 0) and np.all(d[1] == 0)          # env without nodes
    assert (ref.a[2] > 0.1).any()                             # the sensor inside a Gaussian sees it
    d2, a2 = _trace(ds, se, sp, dirs, r_min=50.0, r_max=60.0, build=False, r=r)
    assert np.all(a2 == 0) and np.all(d2 == 0)
    d3, a3 = _trace(ds, se[:0], sp[:0], dirs, build=False, r=r)          # no sensors: nothing to do
    assert d3.size == 0 and a3.size == 0
    r.close()


def test_rebuild_after_attribute_change_and_determinism():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config1(seed=4, n_bg=3000, n_obj=1000)
    ds = DeviceScene(sc, device="cuda:0")
    se, sp = S.lidar_sensors(4, sc.n_envs)
    dirs = S.lidar_pattern(8, 128)
    r = Renderer()
    d0, a0 = _trace(ds, se, sp, dirs, r=r)
    d1, a1 = _trace(ds, se, sp, dirs, r=r, build=False)
    assert np.array_equal(d0, d1) and np.array_equal(a0, a1)
    # halve every opacity in place: stale until rebuilt
    for t, nd in zip(ds.tensors, sc.nodes):
        t["opacity_logit"].sub_(1.0)
        nd.opacity_logit = (nd.opacity_logit - np.float32(1.0)).astype(np.float32)
    d2, a2 = _trace(ds, se, sp, dirs, r=r)
    _check(d2, a2, _oracle(sc, se, sp, dirs), "rebuilt")
    assert not np.array_equal(a2, a0)
    r.close()


def test_full_benchmark_batch_sampled_rays():
    """64 sensors x 32 x 1024 rays through the benchmark scene (1M-Gaussian room + 4 x 20k objects
    per env, Z-ordered), traced in one call; 4 sensors x 384 sampled rays against the oracle and
    sanity on every ray."""
    from paper_2507_21981_gb300.render import DeviceScene
    sc = S.config2(seed=1)
    ds = DeviceScene(sc, device="cuda:0", spatial_order=True)
    se, sp = S.lidar_sensors(1, sc.n_envs)
    dirs = S.lidar_pattern(32, 1024)
    d, a = _trace(ds, se, sp, dirs)
    assert np.isfinite(d).all() and np.isfinite(a).all()
    assert (a >= 0).all() and (a <= 1).all() and (d >= 0).all()
    hit = a > 1e-3
    rng_ = d[hit] / a[hit]
    assert (rng_ >= 0.05 * 0.999).all() and (rng_ <= 30.0 * 1.001).all()
    assert (a > 0.5).mean() > 0.8
    rng = np.random.default_rng(2)
    pk = OO._Packed(ds.scene)
    for s in rng.choice(sc.n_envs, 4, replace=False):
        js = np.sort(rng.choice(len(dirs), 384, replace=False))
        ref = OL.trace(ds.scene, se[s:s + 1], sp[s:s + 1], dirs[js], OL.LidarOptions(), packed=pk)
        _check(d[s:s + 1, js], a[s:s + 1, js], ref, f"full sensor {s}")
