"""Pins of the LiDAR oracle (oracle/lidar.cpp) against facts that do not come from it: the
closed form of an isotropic Gaussian on a ray, the peak of an anisotropic one found by
numerical minimisation (covariance from scipy's rotations), compositing closed forms with
termination, the 3-sigma and range windows, the node pose against pre-transformed Gaussians,
rigid-motion invariance, a brute force on a small random scene that locates each peak by
sampling q(t) along the ray, and exact ties on the decision thresholds whose two closed-form
outcomes must both lie inside the tolerance the oracle returns.  No GPU is needed.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar
from scipy.spatial.transform import Rotation

from oracle import lidar as OL
from paper_2507_21981_gb300 import scenes as S

LO = OL.LidarOptions(r_min=0.05, r_max=30.0, nthreads=2)


def _node(mean, log_scale, quat, logit):
    f = np.float32
    n = len(mean)
    return S.GaussianNode(np.asarray(mean, f).reshape(n, 3), np.asarray(log_scale, f).reshape(n, 3),
                          np.asarray(quat, f).reshape(n, 4), np.asarray(logit, f).reshape(n),
                          np.zeros((n, 1, 3), f), 0, "n")


def _scene(nodes, poses=None):
    poses = poses if poses is not None else [np.eye(3, 4) for _ in nodes]
    return S.scene_from_lists("t", nodes, [list(range(len(nodes)))], [poses],
                              [[(100.0, 100.0, 32.0, 32.0, 64, 64, np.eye(3, 4))]])


def _logit(p):
    return math.log(p / (1 - p))


def _trace(sc, pose, dirs, opts=LO):
    return OL.trace(sc, np.zeros(1, np.int32), np.asarray(pose, np.float64)[None], np.asarray(dirs, np.float64), opts)


def test_isotropic_gaussian_closed_form():
    """A sphere of standard deviation s at mu: the density along the ray peaks at the foot of
    the perpendicular, t* = (mu - o).d, with q* = b^2 / s^2 (b = distance of mu from the ray)."""
    s, op = 0.05, 0.7
    mu = np.array([2.0, 0.3, -0.1], np.float32)
    sc = _scene([_node([mu], [[math.log(s)] * 3], [[1, 0, 0, 0]], [_logit(op)])])
    pose = np.eye(3, 4)
    pose[:, 3] = [0.1, 0.2, 0.0]
    rng = np.random.default_rng(0)
    dirs = mu.astype(np.float64) - pose[:, 3] + rng.normal(0, 0.1, size=(50, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = _trace(sc, pose, dirs)
    s = math.exp(float(np.float32(math.log(s))))              # the values the scene stores (FP32)
    op = 1 / (1 + math.exp(-float(np.float32(_logit(op)))))
    v = mu.astype(np.float64) - pose[:, 3]
    t = dirs @ v
    b2 = np.sum(v * v) - t * t
    q = b2 / s ** 2
    alpha = np.minimum(0.99, op * np.exp(-q / 2))
    hit = (q <= 9) & (alpha >= 1 / 255)
    assert hit.sum() > 10 and (~hit).sum() > 3
    np.testing.assert_allclose(r.a[0], np.where(hit, alpha, 0.0), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r.d[0], np.where(hit, alpha * t, 0.0), rtol=1e-12, atol=1e-15)


def test_anisotropic_gaussian_peak_by_minimisation():
    rng = np.random.default_rng(1)
    for trial in range(10):
        q_xyzw = Rotation.random(random_state=trial).as_quat()
        quat = np.array([q_xyzw[3], *q_xyzw[:3]])
        ls = rng.uniform(-4, -1.5, 3)
        mu = rng.uniform(-1, 1, 3) + np.array([3.0, 0, 0])
        sc = _scene([_node([mu], [ls], [quat], [_logit(0.8)])])
        Rm = Rotation.from_quat(np.asarray(np.float32(q_xyzw), np.float64)).as_matrix()
        Sig_inv = np.linalg.inv(Rm @ np.diag(np.exp(2 * ls.astype(np.float32).astype(np.float64))) @ Rm.T)
        mu64 = mu.astype(np.float32).astype(np.float64)
        o = np.zeros(3)
        d = mu64 - o + rng.normal(0, 0.3 * np.exp(ls).max(), 3)
        d /= np.linalg.norm(d)
        r = _trace(sc, np.eye(3, 4), d[None])

        def qf(t):
            x = o + t * d - mu64
            return x @ Sig_inv @ x
        res = minimize_scalar(qf, bounds=(0.0, 10.0), method="bounded", options={"xatol": 1e-12})
        q_min = qf(res.x)
        alpha = min(0.99, 0.8 * math.exp(-q_min / 2))
        if q_min <= 9 and alpha >= 1 / 255:
            assert r.a[0, 0] == pytest.approx(alpha, rel=1e-7)
            assert r.d[0, 0] / r.a[0, 0] == pytest.approx(res.x, abs=1e-6)
        else:
            assert r.a[0, 0] == 0.0


def test_compositing_two_and_three_gaussians():
    """Front-to-back over the hits in order of t*: D = a1 t1 + (1 - a1) a2 t2; with three
    opaque (0.99) Gaussians the third would drive T to 1e-6 < t_min and is not composited.
    (Opacity logits are stored in FP32: the opacities match to 1e-7.)"""
    sc = _scene([_node([[4.0, 0, 0], [2.0, 0, 0]], [[-3] * 3] * 2, [[1, 0, 0, 0]] * 2, [_logit(0.5), _logit(0.3)])])
    r = _trace(sc, np.eye(3, 4), [[1.0, 0, 0]])
    assert r.d[0, 0] == pytest.approx(0.3 * 2 + 0.7 * 0.5 * 4, rel=1e-7)
    assert r.a[0, 0] == pytest.approx(1 - 0.7 * 0.5, rel=1e-7)
    big = _logit(0.999)
    sc = _scene([_node([[3.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]], [[-3] * 3] * 3, [[1, 0, 0, 0]] * 3, [big] * 3)])
    r = _trace(sc, np.eye(3, 4), [[1.0, 0, 0]])
    assert r.d[0, 0] == pytest.approx(0.99 * 1 + 0.01 * 0.99 * 2, rel=1e-7)
    assert r.a[0, 0] == pytest.approx(1 - 1e-4, rel=1e-7)
    assert r.n_comp[0, 0] == 2


def test_three_sigma_and_range_windows():
    s = 0.1
    mus = [[2.0, 2.99 * s, 0], [2.5, 3.01 * s, 0], [0.03, 0, 0], [31.0, 0, 0], [-2.0, 0, 0]]
    sc = _scene([_node(mus, [[math.log(s)] * 3] * 5, [[1, 0, 0, 0]] * 5, [_logit(0.9)] * 5)])
    r = _trace(sc, np.eye(3, 4), [[1.0, 0, 0]])
    # only the first: the second is outside 3 sigma, the third before r_min, the fourth beyond
    # r_max, the fifth behind the sensor
    a1 = 0.9 * math.exp(-0.5 * 2.99 ** 2)
    assert r.a[0, 0] == pytest.approx(a1, rel=1e-5)
    assert r.d[0, 0] == pytest.approx(a1 * 2.0, rel=1e-5)


def _rand_node(rng, n, centre, spread):
    q = Rotation.random(n, random_state=int(rng.integers(1 << 30))).as_quat()
    return _node(centre + rng.uniform(-spread, spread, (n, 3)), rng.uniform(-3.5, -2.0, (n, 3)),
                 np.concatenate([q[:, 3:], q[:, :3]], axis=1), rng.normal(0.5, 1.0, n))


def test_node_pose_equals_pretransformed_gaussians():
    rng = np.random.default_rng(3)
    nd = _rand_node(rng, 60, np.zeros(3), 0.4)
    P = S.random_pose(rng, 0.5)
    P[:, 3] += [3.0, 0.0, 0.0]
    R = P[:, :3]
    mean_w = nd.mean.astype(np.float64) @ R.T + P[:, 3]
    q_n = np.asarray(nd.quat, np.float64)
    rot = Rotation.from_matrix(R) * Rotation.from_quat(np.concatenate([q_n[:, 1:], q_n[:, :1]], axis=1))
    qw = rot.as_quat()
    nd_w = _node(mean_w, nd.log_scale, np.concatenate([qw[:, 3:], qw[:, :3]], axis=1), nd.opacity_logit)
    dirs = S.lidar_pattern(16, 64, -20, 20)
    a = _trace(_scene([nd], [P]), np.eye(3, 4), dirs)
    b = _trace(_scene([nd_w]), np.eye(3, 4), dirs)
    # the pre-transformed scene is rounded to FP32: compare within its tolerance
    assert (a.a > 0.05).sum() > 20
    np.testing.assert_allclose(a.a, b.a, atol=2e-5)
    np.testing.assert_allclose(a.d, b.d, atol=1e-4)


def test_rigid_motion_invariance():
    rng = np.random.default_rng(4)
    nodes = [_rand_node(rng, 80, np.array([2.0, 0, 0]), 0.6), _rand_node(rng, 30, np.zeros(3), 0.2)]
    P1 = S.random_pose(rng, 0.3)
    P1[:, 3] += [2.0, 0.5, 0.0]
    poses = [np.eye(3, 4), P1]
    sensor = np.eye(3, 4)
    sensor[:, 3] = [-0.5, 0.1, 0.0]
    dirs = S.lidar_pattern(8, 48, -25, 25)
    r0 = _trace(_scene(nodes, poses), sensor, dirs)
    G = S.random_pose(rng, 2.0)

    def compose(A, B):
        return np.concatenate([A[:, :3] @ B[:, :3], (A[:, :3] @ B[:, 3] + A[:, 3])[:, None]], axis=1)
    r1 = OL.trace(_scene(nodes, [compose(G, p) for p in poses]), np.zeros(1, np.int32),
                  compose(G, sensor)[None], dirs, LO)
    # poses and sensor are FP64 here; the scene stores node poses in FP32
    assert (r0.a > 0.05).sum() > 10
    np.testing.assert_allclose(r1.a, r0.a, atol=1e-5)
    np.testing.assert_allclose(r1.d, r0.d, atol=1e-4)


def test_brute_force_by_sampling_small_scene():
    """Every Gaussian's peak located by dense sampling of q(t) on the ray and refined by a
    bounded scalar minimisation; hits sorted by (t, id) and composited."""
    rng = np.random.default_rng(5)
    nodes = [_rand_node(rng, 25, np.array([2.0, 0, 0]), 0.3), _rand_node(rng, 15, np.zeros(3), 0.15)]
    P1 = S.random_pose(rng, 0.1)
    P1[:, 3] += [1.6, 0.0, 0.05]
    sc = _scene(nodes, [np.eye(3, 4), P1])
    dirs = S.lidar_pattern(6, 24, -15, 15, az0_deg=-30, az_span_deg=60).astype(np.float64)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = _trace(sc, np.eye(3, 4), dirs)
    gs = []
    for k, (nd, P) in enumerate(zip(nodes, [np.eye(3, 4), P1])):
        P = np.asarray(P, np.float32).astype(np.float64)
        for i in range(nd.n):
            q = np.asarray(nd.quat[i], np.float64)
            Rm = P[:, :3] @ Rotation.from_quat([*q[1:], q[0]]).as_matrix()
            Sig = Rm @ np.diag(np.exp(2 * np.asarray(nd.log_scale[i], np.float64))) @ Rm.T
            mu = P[:, :3] @ np.asarray(nd.mean[i], np.float64) + P[:, 3]
            op = 1 / (1 + math.exp(-float(nd.opacity_logit[i])))
            gs.append((mu, np.linalg.inv(Sig), op, len(gs)))
    ts = np.linspace(0.0, 30.0, 30001)
    n_hit = 0
    for j, d in enumerate(dirs):
        hits = []
        for mu, Si, op, gid in gs:
            x = ts[:, None] * d[None, :] - mu[None, :]
            qs = np.einsum("ni,ij,nj->n", x, Si, x)
            k = int(np.argmin(qs))
            lo, hi = ts[max(k - 1, 0)], ts[min(k + 1, len(ts) - 1)]
            res = minimize_scalar(lambda t: (t * d - mu) @ Si @ (t * d - mu), bounds=(lo, hi), method="bounded",
                                  options={"xatol": 1e-12})
            qm = (res.x * d - mu) @ Si @ (res.x * d - mu)
            a = min(0.99, op * math.exp(-qm / 2))
            if qm <= 9 and 0.05 <= res.x <= 30 and a >= 1 / 255:
                hits.append((res.x, gid, a))
        hits.sort()
        T, D = 1.0, 0.0
        for t, _, a in hits:
            if T * (1 - a) < 1e-4:
                break
            D += T * a * t
            T *= 1 - a
        n_hit += bool(hits)
        assert r.a[0, j] == pytest.approx(1 - T, abs=1e-6)
        assert r.d[0, j] == pytest.approx(D, abs=1e-5)
    assert n_hit > 20


def test_tolerance_is_tight_on_a_room():
    """On the room workload the derived FP32 tolerance stays small for most rays: it cannot be
    hiding gross errors (missing one surface Gaussian of opacity > 0.05 exceeds it)."""
    sc = S.config2(seed=1, n_envs=1, n_bg=60_000, n_obj=2_000)
    se, sp = S.lidar_sensors(1, 1)
    r = OL.trace(sc, se, sp, S.lidar_pattern(8, 128), OL.LidarOptions())
    hit = r.a > 0.5
    assert hit.mean() > 0.25           # a sparse room (60k Gaussians): many rays pass through
    # thin surface Gaussians (1.8 mm normal axis) make FP32 positions at metres the main error
    assert np.median(r.tol_a[hit]) < 3e-3 and np.median(r.tol_d[hit] / r.d[hit]) < 3e-3


def test_tolerance_rejects_plausible_mistakes():
    """The per-ray tolerance the GPU is held to is tight enough to catch plausible mistakes:
    ignoring the node poses, Gaussians 5 % too large, and a sensor 1 mm off along its beams each
    move D or A beyond twice the tolerance on many rays of a posed multi-node scene."""
    rng = np.random.default_rng(8)
    nodes = [_rand_node(rng, 400, np.array([2.0, 0, 0]), 0.5), _rand_node(rng, 200, np.zeros(3), 0.2)]
    P1 = S.random_pose(rng, 0.3)
    P1[:, 3] += [1.8, 0.3, 0.0]
    poses = [np.eye(3, 4), P1]
    dirs = S.lidar_pattern(16, 64, -25, 25, az0_deg=-40, az_span_deg=80).astype(np.float64)
    sensor = np.eye(3, 4)
    ref = _trace(_scene(nodes, poses), sensor, dirs)
    hit = ref.a > 0.05
    assert hit.sum() > 100

    def frac_beyond(other):
        bad = (np.abs(other.a - ref.a) > 2 * ref.tol_a + 1e-6) | (np.abs(other.d - ref.d) > 2 * ref.tol_d + 1e-6)
        return float(bad[hit].mean())
    no_pose = _trace(_scene(nodes, [np.eye(3, 4), np.eye(3, 4)]), sensor, dirs)
    big = [_node(nd.mean, nd.log_scale + np.float32(np.log(1.05)), nd.quat, nd.opacity_logit) for nd in nodes]
    bigger = _trace(_scene(big, poses), sensor, dirs)
    moved = sensor.copy()
    moved[:, 3] = [0.001, 0.0, 0.0]
    shifted = _trace(_scene(nodes, poses), moved, dirs)
    assert frac_beyond(no_pose) > 0.8           # measured: 100 %, 99.6 % and 99.4 % of hit rays
    assert frac_beyond(bigger) > 0.8
    assert frac_beyond(shifted) > 0.8


# The FP32 tracer may take either side of a decision that lies on its threshold.  Each case
# puts one decision exactly there, on a ray along +x from the origin through isotropic
# Gaussians (s = 0.1, identity rotation), and checks that the oracle flags it and that both
# closed-form outcomes lie within the tolerance it returns around its primary result.
def _tie(mus, logits, opts=LO):
    n = len(mus)
    sc = _scene([_node(mus, [[math.log(0.1)] * 3] * n, [[1, 0, 0, 0]] * n, logits)])
    return _trace(sc, np.eye(3, 4), [[1.0, 0, 0]], opts)


def _covers(r, outcomes):
    assert r.n_amb[0, 0] >= 1
    for a, d in outcomes:
        assert abs(a - r.a[0, 0]) <= r.tol_a[0, 0] + 1e-12, (a, r.a[0, 0], r.tol_a[0, 0])
        assert abs(d - r.d[0, 0]) <= r.tol_d[0, 0] + 1e-12, (d, r.d[0, 0], r.tol_d[0, 0])


def _f32(x):
    return float(np.float32(x))


def _alpha(y, logit):
    """Closed form on the stored FP32 inputs: opacity sigmoid(logit) times exp(-q*/2), q* the
    squared perpendicular distance y over s."""
    s = math.exp(_f32(math.log(0.1)))
    return math.exp(-0.5 * (_f32(y) / s) ** 2) / (1 + math.exp(-_f32(logit)))


def test_tie_on_the_three_sigma_ellipsoid():
    a9 = _alpha(0.3, _logit(0.9))             # perpendicular distance 3 s: q* = 9
    _covers(_tie([[2.0, 0.3, 0.0]], [_logit(0.9)]), [(0.0, 0.0), (a9, a9 * 2.0)])


def test_tie_on_the_far_end_of_the_range_window():
    a = _alpha(0.0, _logit(0.9))
    _covers(_tie([[30.0, 0.0, 0.0]], [_logit(0.9)]), [(0.0, 0.0), (a, a * 30.0)])


def test_tie_on_alpha_min():
    a = _alpha(0.0, _logit(1 / 255))           # 1/255 up to the FP32 rounding of the logit
    assert a == pytest.approx(1 / 255, rel=1e-6)
    _covers(_tie([[2.0, 0.0, 0.0]], [_logit(1 / 255)]), [(0.0, 0.0), (a, a * 2.0)])


def test_tie_on_the_termination_threshold():
    # two hits clamped at alpha 0.99: T = 0.01, then 0.01 * 0.01 = t_min
    r = _tie([[2.0, 0.0, 0.0], [3.0, 0.0, 0.0]], [10.0, 10.0])
    _covers(r, [(0.99, 0.99 * 2.0), (1 - 1e-4, 0.99 * 2.0 + 0.0099 * 3.0)])


def test_decisions_away_from_thresholds_are_not_flagged():
    """Control for the ties above: 2.5 s off the ray, alpha well above alpha_min, well inside
    the window and far from t_min, nothing is flagged and the tolerance is far below the hit's
    own weight."""
    a = 0.9 * math.exp(-0.5 * 2.5 ** 2)
    r = _tie([[2.0, 0.25, 0.0]], [_logit(0.9)])
    assert r.n_amb[0, 0] == 0
    assert r.a[0, 0] == pytest.approx(a, rel=1e-5) and r.tol_a[0, 0] < 1e-3 * a and r.tol_d[0, 0] < 1e-3 * a * 2.0
