"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test states what fixes the expected value: a library routine (scipy's complex spherical
harmonics, scipy's rotation matrices), a closed form of the EWA projection of an isotropic
Gaussian, compositing invariants (weights + transmittance = 1), rigid-motion invariance,
brute force, finite differences, or the two closed-form outcomes of a decision placed exactly
on its threshold.  No GPU is needed.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

import oracle as O
from paper_2507_21981_gb300 import scenes as S
from tests import scene_utils as U

BASE = O.OracleOptions(nthreads=4)


def opts(**kw):
    d = dict(BASE.__dict__)
    d.update(kw)
    return O.OracleOptions(**d)


# --------------------------------------------------------------------------- spherical harmonics
def _real_sh_scipy(l, m, d):
    """Real SH with the Condon-Shortley phase from scipy's complex Y_l^m (which includes it)."""
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0]) % (2 * math.pi)
    if m == 0:
        return sph_harm_y(l, 0, theta, phi).real
    Y = sph_harm_y(l, abs(m), theta, phi)
    return math.sqrt(2) * (Y.real if m > 0 else Y.imag)


def test_sh_matches_scipy_complex_harmonics():
    rng = np.random.default_rng(0)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y, _ = O.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert Y[l * l + l + m] == pytest.approx(_real_sh_scipy(l, m, d), abs=1e-13)


def test_sh_degree_one_closed_form():
    rng = np.random.default_rng(1)
    c = math.sqrt(3 / (4 * math.pi))
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y, _ = O.sh_basis(1, d)
        np.testing.assert_allclose(Y[1:4], c * np.array([-d[1], d[2], -d[0]]), atol=1e-15)
        assert np.all(Y[4:] == 0)


def test_sh_orthonormal_on_sphere():
    # Gauss-Legendre in z (exact to degree 15) x uniform azimuth (exact for |m| <= 7).
    zs, wz = np.polynomial.legendre.leggauss(8)
    phis = np.arange(16) * 2 * np.pi / 16
    Gram = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        r = math.sqrt(1 - z * z)
        for ph in phis:
            Y, _ = O.sh_basis(3, np.array([r * math.cos(ph), r * math.sin(ph), z]))
            Gram += w * (2 * np.pi / 16) * np.outer(Y, Y)
    np.testing.assert_allclose(Gram, np.eye(16), atol=1e-13)


def test_sh_tangential_gradient_matches_fd():
    rng = np.random.default_rng(2)
    for _ in range(10):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        _, dY = O.sh_basis(3, d)
        P = np.eye(3) - np.outer(d, d)
        for j in range(3):
            h = 1e-6
            e = np.zeros(3); e[j] = h
            Yp, _ = O.sh_basis(3, (d + e) / np.linalg.norm(d + e))
            Ym, _ = O.sh_basis(3, (d - e) / np.linalg.norm(d - e))
            fd = (Yp - Ym) / (2 * h)
            np.testing.assert_allclose((dY @ P)[:, j], fd, atol=1e-8)


def test_degree_zero_colour_is_view_independent():
    rng = np.random.default_rng(3)
    nd = U.node([[0, 0, 5.0]], sh=U.colour_sh([[0.2, 0.6, 0.9]]), deg=0)
    for _ in range(5):
        cam = U.rigid(Rotation.random(random_state=rng).as_matrix(), rng.normal(size=3))
        # place the camera so the Gaussian is in front of it: move it along its own z axis
        R = cam[:, :3]
        centre = np.array([0, 0, 5.0]) - 3.0 * R[2]
        cam = U.rigid(R, -R @ centre)
        sc = U.single_view([nd], cam=cam)
        p = O.project_view(sc, 0, 0, BASE)
        np.testing.assert_allclose(p[0, 11:14], [0.2, 0.6, 0.9], atol=1e-7)


def test_colour_uses_node_frame_direction():
    """Rotating a node together with the camera leaves its SH colour unchanged."""
    rng = np.random.default_rng(4)
    sh = rng.normal(0, 0.2, (1, 16, 3))
    nd = U.node([[0.1, -0.2, 0.3]], sh=sh, deg=3, dtype=np.float64)
    cam0 = U.rigid(np.eye(3), [0, 0, 4.0])
    base = O.project_view(U.single_view([nd], cam=cam0), 0, 0, BASE)[0, 11:14]
    for _ in range(5):
        G = U.rigid(Rotation.random(random_state=rng).as_matrix(), rng.normal(size=3))
        sc = U.single_view([nd], poses=[G], cam=U.compose(cam0, U.inverse(G)))
        np.testing.assert_allclose(O.project_view(sc, 0, 0, BASE)[0, 11:14], base, atol=1e-12)


# --------------------------------------------------------------------------- projection
@pytest.mark.parametrize("lowpass", [0.0, 0.3])
def test_isotropic_projection_closed_form(lowpass):
    sigma, f = 0.05, 60.0
    pts = [[0.0, 0.0, 4.0], [0.5, -0.3, 3.0], [-0.8, 0.6, 5.0]]
    nd = U.node(pts, log_scales=np.full((3, 3), math.log(sigma)), dtype=np.float64)
    sc = U.single_view([nd], f=f, W=64, H=64, cx=32.0, cy=30.0)
    p = O.project_view(sc, 0, 0, opts(lowpass=lowpass))
    assert p.shape[0] == 3
    for row, (x, y, z) in zip(p, pts):
        # J J^T sigma^2 for J = f/z [[1, 0, -x/z], [0, 1, -y/z]]
        k = (f * sigma / z) ** 2
        cov = k * np.array([[1 + x * x / z / z, x * y / z / z], [x * y / z / z, 1 + y * y / z / z]]) + lowpass * np.eye(2)
        np.testing.assert_allclose(row[[7, 8, 9]], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-12)
        inv = np.linalg.inv(cov)
        np.testing.assert_allclose(row[[4, 5, 6]], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-11)
        np.testing.assert_allclose(row[[1, 2, 3]], [f * x / z + 32.0, f * y / z + 30.0, z], rtol=1e-14)


def test_anisotropic_projection_matches_rotation_library():
    rng = np.random.default_rng(5)
    n = 20
    q = rng.normal(size=(n, 4))                       # (w,x,y,z), not normalised
    ls = rng.normal(-2.5, 0.5, (n, 3))
    mu = rng.uniform(-0.5, 0.5, (n, 3))
    nd = U.node(mu, log_scales=ls, quats=q, dtype=np.float64)
    pose = U.rigid(Rotation.random(random_state=rng).as_matrix(), [0.1, 0.2, 0.3])
    cam = U.rigid(np.eye(3), [0, 0, 3.0])
    fx = 80.0
    sc = U.single_view([nd], poses=[pose], cam=cam, f=fx, W=96, H=96)
    p = O.project_view(sc, 0, 0, opts(lowpass=0.0))
    assert p.shape[0] == n
    for row in p:
        g = int(row[0])
        R = Rotation.from_quat([q[g, 1], q[g, 2], q[g, 3], q[g, 0]]).as_matrix()   # scipy is scalar-last
        Sig = R @ np.diag(np.exp(2 * ls[g])) @ R.T
        Rn, tn = pose[:, :3], pose[:, 3]
        t = cam[:, :3] @ (Rn @ mu[g] + tn) + cam[:, 3]
        J = np.array([[fx / t[2], 0, -fx * t[0] / t[2] ** 2], [0, fx / t[2], -fx * t[1] / t[2] ** 2]])
        Tm = J @ cam[:, :3] @ Rn
        cov = Tm @ Sig @ Tm.T
        np.testing.assert_allclose(row[[7, 8, 9]], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-10, atol=1e-14)


# --------------------------------------------------------------------------- compositing
def test_peak_alpha_at_centre_pixel():
    for logit, expect in [(0.3, 1 / (1 + math.exp(-0.3))), (8.0, 0.99), (-2.0, 1 / (1 + math.exp(2.0)))]:
        nd = U.node([[0.0, 0.0, 4.0]], logits=[logit], sh=U.colour_sh([[0.7, 0.2, 0.4]]))
        sc = U.single_view([nd], W=32, H=32, cx=16.5, cy=16.5)        # centre lands on pixel (16,16)
        for bg in [(0, 0, 0), (0.1, 0.5, 1.0)]:
            r = O.render_view(sc, 0, 0, opts(bg=bg))
            a = r.alpha[16, 16]
            assert a == pytest.approx(min(0.99, expect), rel=1e-7)      # logits are stored as float32
            colour = np.array([0.7, 0.2, 0.4], np.float32).astype(np.float64)
            np.testing.assert_allclose(r.rgb[16, 16], colour * a + (1 - a) * np.array(bg), rtol=1e-6)


def test_single_gaussian_closed_form_image():
    sigma, f, z, opac = 0.08, 50.0, 4.0, 0.8
    nd = U.node([[0.0, 0.0, z]], log_scales=np.full((1, 3), math.log(sigma)), logits=[math.log(opac / (1 - opac))],
                sh=U.colour_sh([[0.3, 0.6, 0.9]]), dtype=np.float64)
    sc = U.single_view([nd], f=f, W=24, H=24, cx=12.0, cy=12.0)
    lp = 0.3
    r = O.render_view(sc, 0, 0, opts(lowpass=lp, bg=(0.2, 0.2, 0.2)))
    s2 = (f * sigma / z) ** 2 + lp
    ys, xs = np.mgrid[0:24, 0:24]
    q = ((xs + 0.5 - 12.0) ** 2 + (ys + 0.5 - 12.0) ** 2) / s2
    a = np.minimum(0.99, opac * np.exp(-0.5 * q))
    keep = (q <= 9) & (a >= 1 / 255)
    a = np.where(keep, a, 0)
    np.testing.assert_allclose(r.alpha, a, atol=1e-13)
    np.testing.assert_allclose(r.depth, a * z, atol=1e-12)
    np.testing.assert_allclose(r.rgb, a[..., None] * [0.3, 0.6, 0.9] + (1 - a[..., None]) * 0.2, atol=1e-12)


def test_weights_and_transmittance_sum_to_one():
    sc = S.config1(seed=7, n_bg=600, n_obj=150, res=48, f=41.25)
    for nd in sc.nodes:
        nd.sh[:] = U.colour_sh([[1.0, 1.0, 1.0]])[0]
    r0 = O.render_view(sc, 0, 0, opts(bg=(0, 0, 0)))
    r1 = O.render_view(sc, 0, 0, opts(bg=(1, 1, 1)))
    assert r0.alpha.max() > 0.5
    for ch in range(3):
        np.testing.assert_allclose(r0.rgb[..., ch], r0.alpha, atol=1e-12)
        np.testing.assert_allclose(r1.rgb[..., ch], 1.0, atol=1e-12)


def test_depth_of_a_fronto_parallel_layer():
    rng = np.random.default_rng(8)
    z = 3.0
    mu = np.c_[rng.uniform(-0.6, 0.6, (80, 2)), np.full(80, z)]
    nd = U.node(mu, log_scales=rng.normal(-2.5, 0.3, (80, 3)), logits=rng.normal(0, 1, 80),
                sh=U.colour_sh(rng.random((80, 3))))
    sc = U.single_view([nd], f=40.0)
    r = O.render_view(sc, 0, 0, BASE)
    np.testing.assert_allclose(r.depth, z * r.alpha, rtol=1e-12, atol=1e-14)


def test_termination_stops_without_compositing():
    # four coincident-footprint Gaussians on the axis at increasing depth, alpha 0.95 each at
    # the centre pixel: T = 1, .05, .0025, 1.25e-4, then 6.25e-6 < 1e-4 -> stop before the 4th.
    cols = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], np.float64)
    logit = math.log(0.95 / 0.05)
    nd = U.node([[0, 0, 3.0], [0, 0, 3.1], [0, 0, 3.2], [0, 0, 3.3]], log_scales=np.full((4, 3), math.log(0.3)),
                logits=[logit] * 4, sh=U.colour_sh(cols), dtype=np.float64)
    sc = U.single_view([nd], W=16, H=16, cx=8.5, cy=8.5)
    r = O.render_view(sc, 0, 0, opts(bg=(0.5, 0.5, 0.5)))
    T, C, D = 1.0, np.zeros(3), 0.0
    for i in range(3):
        C += 0.95 * T * cols[i]; D += 0.95 * T * [3.0, 3.1, 3.2][i]; T *= 0.05
    np.testing.assert_allclose(r.rgb[8, 8], C + 0.5 * T, rtol=1e-12)
    assert r.depth[8, 8] == pytest.approx(D, rel=1e-12)
    assert r.alpha[8, 8] == pytest.approx(1 - T, rel=1e-12)


def test_faint_gaussian_is_skipped_not_terminal():
    nd = U.node([[0, 0, 3.0], [0, 0, 4.0]], log_scales=np.full((2, 3), math.log(0.3)),
                logits=[math.log(0.003 / 0.997), 1.0], sh=U.colour_sh([[1, 0, 0], [0, 1, 0]]), dtype=np.float64)
    sc = U.single_view([nd], W=16, H=16, cx=8.5, cy=8.5)
    r = O.render_view(sc, 0, 0, BASE)
    a = 1 / (1 + math.exp(-1.0))
    np.testing.assert_allclose(r.rgb[8, 8], [0, a, 0], atol=1e-12)


def test_storage_order_does_not_matter_for_distinct_depths():
    sc = S.config1(seed=9, n_bg=300, n_obj=100, res=32, f=27.5)
    r = O.render_view(sc, 0, 0, BASE)
    swapped = S.scene_from_lists("swap", [sc.nodes[1], sc.nodes[0]], [[0, 1]],
                                 [[sc.node_poses[0, 1], sc.node_poses[0, 0]]],
                                 [[(*sc.cam_intr[0, 0], *sc.cam_res[0, 0], sc.cam_pose[0, 0])]])
    r2 = O.render_view(swapped, 0, 0, BASE)
    np.testing.assert_allclose(r2.rgb, r.rgb, atol=1e-13)
    np.testing.assert_allclose(r2.depth, r.depth, atol=1e-13)


def test_zero_opacity_gives_background():
    sc = S.config1(seed=10, n_bg=200, n_obj=50, res=32, f=27.5)
    for nd in sc.nodes:
        nd.opacity_logit[:] = -40.0
    r = O.render_view(sc, 0, 0, opts(bg=(0.25, 0.5, 0.75)))
    np.testing.assert_allclose(r.rgb, np.broadcast_to([0.25, 0.5, 0.75], r.rgb.shape), atol=0)
    assert np.all(r.depth == 0) and np.all(r.alpha == 0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bruteforce_agrees_with_candidate_lists(seed):
    sc = S.config1(seed=seed, n_bg=40, n_obj=10, res=16, f=13.75)
    a = O.render_view(sc, 0, 0, BASE)
    b = O.render_view(sc, 0, 0, opts(bruteforce=1))
    assert a.instances == b.instances
    assert np.array_equal(a.rgb, b.rgb) and np.array_equal(a.depth, b.depth) and np.array_equal(a.alpha, b.alpha)
    assert a.decision_hash == b.decision_hash


def test_bruteforce_agrees_on_fd_subset():
    sc = S.fd_subset(seed=4)
    a = O.render_view(sc, 0, 0, BASE)
    b = O.render_view(sc, 0, 0, opts(bruteforce=1))
    assert np.array_equal(a.rgb, b.rgb) and np.array_equal(a.depth, b.depth)


def test_rigid_motion_of_scene_and_camera_leaves_image_unchanged():
    rng = np.random.default_rng(11)
    sc = S.config1(seed=11, n_bg=800, n_obj=200, res=40, f=34.4)
    o = BASE
    r = O.render_view(sc, 0, 0, o)
    for _ in range(3):
        G = U.rigid(Rotation.random(random_state=rng).as_matrix(), rng.normal(size=3) * 2)
        poses = np.stack([U.compose(G, sc.node_poses[0, j].astype(np.float64)) for j in range(2)])[None]
        cam = U.compose(sc.cam_pose[0, 0].astype(np.float64), U.inverse(G))[None, None]
        moved = S.Scene("moved", sc.nodes, sc.env_node_ids, poses, sc.cams_per_env, sc.cam_intr, sc.cam_res, cam)
        r2 = O.render_view(moved, 0, 0, o)
        np.testing.assert_allclose(r2.rgb, r.rgb, atol=1e-10)
        np.testing.assert_allclose(r2.depth, r.depth, atol=1e-10)


def test_ambiguity_fraction_is_small_on_config1():
    # pixels with at least one decision inside its FP32 error band (branches checked one by one)
    r = O.render_view(S.config1(seed=1), 0, 0, BASE)
    assert r.ambiguous_pixels / r.rgb[..., 0].size < 2e-2
    assert r.tol_rgb.max() == 0.0          # no pixel needed more than max_flips branches


def test_empty_node_and_empty_env_render_background():
    sc = S.config1(seed=12, n_bg=100, n_obj=30, res=16, f=13.75)
    sc.nodes[1] = sc.nodes[1].subset(slice(0, 0))
    r = O.render_view(sc, 0, 0, opts(bg=(0.5, 0.5, 0.5)))
    assert r.instances <= 100
    sc.env_node_ids[0, :] = -1
    r = O.render_view(sc, 0, 0, opts(bg=(0.5, 0.5, 0.5)))
    assert r.instances == 0 and np.all(r.rgb == 0.5) and np.all(r.depth == 0)


# --------------------------------------------------------------------------- FP32-ambiguous decisions
# The method's cutoffs (Sec. III-A compositing: alpha below 1/255 skipped, stop once T < 1e-4,
# the 3-sigma ellipse) are thresholds an FP32 evaluation may land on either side of.  Each case
# places one decision exactly on its threshold in a hand-built scene whose two outcomes have
# closed forms; the oracle must flag that pixel and return both branches.
def _branches(r, y, x):
    """Every branch's (r, g, b, d, a) at pixel (y, x): the primary result, then the alternatives."""
    p = y * r.rgb.shape[1] + x
    prim = np.r_[r.rgb[y, x], r.depth[y, x], r.alpha[y, x]]
    return np.vstack([prim[None], r.alternatives(p)[:, :5]])


def _same_branches(got, want, tol=1e-12):
    assert len(got) == len(want), (got, want)
    for w in want:
        assert np.abs(got - np.asarray(w)).max(axis=1).min() <= tol, (got, want)


C_FG, C_BG = np.array([0.9, 0.3, 0.1]), np.array([0.2, 0.4, 0.6])


def _alpha_tie_scene():
    # opacity exactly alpha_min; the mean projects onto the centre of pixel (8, 8) (q = 0)
    p = 1 / 255
    nd = U.node([[0, 0, 4.0]], log_scales=np.full((1, 3), math.log(0.08)), logits=[math.log(p / (1 - p))],
                sh=U.colour_sh([C_FG]), dtype=np.float64)
    return U.single_view([nd], f=100.0, W=17, H=17, cx=8.5, cy=8.5), p, 4.0


def test_alpha_min_tie_returns_composited_and_skipped_branches():
    sc, p, z = _alpha_tie_scene()
    r = O.render_view(sc, 0, 0, opts(bg=tuple(C_BG)))
    assert r.ambiguous_by_kind["alpha"] == 1 and r.ambiguous_pixels == 1 and r.n_alt[8, 8] == 1
    _same_branches(_branches(r, 8, 8), [np.r_[p * C_FG + (1 - p) * C_BG, p * z, p], np.r_[C_BG, 0, 0]])


def test_unexplored_flip_widens_the_tolerance_over_the_other_branch():
    sc, p, z = _alpha_tie_scene()
    r = O.render_view(sc, 0, 0, opts(bg=tuple(C_BG), max_flips=0))
    assert r.n_alt[8, 8] == 0 and r.ambiguous_pixels == 1
    comp, skip = np.r_[p * C_FG + (1 - p) * C_BG, p * z], np.r_[C_BG, 0.0]
    other = skip if abs(r.alpha[8, 8]) < 1e-15 else comp                 # the branch not taken
    here = np.r_[r.rgb[8, 8], r.depth[8, 8]]
    assert r.tol_rgb[8, 8] >= np.abs(other[:3] - here[:3]).max() - 1e-15
    assert r.tol_d[8, 8] >= abs(other[3] - here[3]) - 1e-15


def test_transmittance_tie_returns_stop_and_composite_branches():
    # two Gaussians clamped at alpha 0.99 on the centre pixel: T = 0.01, then 0.01 * 0.01 = t_min
    c2 = np.array([0.1, 0.8, 0.5])
    nd = U.node([[0, 0, 3.0], [0, 0, 4.0]], log_scales=np.full((2, 3), math.log(0.3)), logits=[10.0, 10.0],
                sh=U.colour_sh([C_FG, c2]), dtype=np.float64)
    sc = U.single_view([nd], W=17, H=17, cx=8.5, cy=8.5)
    r = O.render_view(sc, 0, 0, opts(bg=tuple(C_BG)))
    assert r.ambiguous_by_kind["transmittance"] >= 1 and r.n_alt[8, 8] == 1
    stop = np.r_[0.99 * C_FG + 0.01 * C_BG, 0.99 * 3.0, 0.99]
    comp = np.r_[0.99 * C_FG + 0.0099 * c2 + 1e-4 * C_BG, 0.99 * 3.0 + 0.0099 * 4.0, 1 - 1e-4]
    _same_branches(_branches(r, 8, 8), [stop, comp])


def test_ellipse_boundary_tie_returns_inside_and_outside_branches():
    # f sigma / z = 1 px and no low-pass: q = (distance in px)^2, so the four pixels 3 px from
    # the centre lie on q_max = 9, where alpha = sigmoid(8) exp(-4.5) is well above alpha_min
    z = 4.0
    nd = U.node([[0, 0, z]], log_scales=np.full((1, 3), math.log(0.04)), logits=[8.0], sh=U.colour_sh([C_FG]),
                dtype=np.float64)
    sc = U.single_view([nd], f=100.0, W=17, H=17, cx=8.5, cy=8.5)
    r = O.render_view(sc, 0, 0, opts(lowpass=0.0, bg=tuple(C_BG)))
    assert r.ambiguous_by_kind["ellipse"] == 4 and r.ambiguous_pixels == 4
    a9 = math.exp(-4.5) / (1 + math.exp(-8.0))
    for y, x in [(8, 11), (8, 5), (11, 8), (5, 8)]:
        assert r.n_alt[y, x] == 1
        _same_branches(_branches(r, y, x), [np.r_[a9 * C_FG + (1 - a9) * C_BG, a9 * z, a9], np.r_[C_BG, 0, 0]])


# --------------------------------------------------------------------------- depth order and near plane
# The method sorts by an FP32 depth key (Sec. III-A depth sorting); the oracle orders by the FP64
# depth, so two Gaussians whose depths differ by less than the FP32 error bands of their depths
# may come in either order, and a centre on the near plane may be culled or kept.
def _two_on_axis(dz_rel, alphas=(0.6, 0.5), cols=(C_FG, np.array([0.1, 0.8, 0.5])), z=4.0):
    logits = [math.log(a / (1 - a)) for a in alphas]
    nd = U.node([[0, 0, z], [0, 0, z * (1 + dz_rel)]], log_scales=np.full((2, 3), math.log(0.08)), logits=logits,
                sh=U.colour_sh(np.asarray(cols)), dtype=np.float64)
    return U.single_view([nd], f=100.0, W=17, H=17, cx=8.5, cy=8.5)


def _composite(seq, bg):
    """Closed-form front-to-back composite of (alpha, colour, z) triples (no cutoff reached)."""
    T, C, D = 1.0, np.zeros(3), 0.0
    for a, c, z in seq:
        C = C + a * T * np.asarray(c)
        D += a * T * z
        T *= 1 - a
    return np.r_[C + T * np.asarray(bg), D, 1 - T]


def test_near_tie_pair_returns_both_orders():
    z, dz_rel = 4.0, 2.5e-8                       # 1e-7 m apart: inside the FP32 bands of the two depths
    c1, c2 = C_FG, np.array([0.1, 0.8, 0.5])
    sc = _two_on_axis(dz_rel, cols=(c1, c2), z=z)
    r = O.render_view(sc, 0, 0, opts(bg=tuple(C_BG)))
    assert r.ambiguous_by_kind["order"] >= 1 and r.n_alt[8, 8] == 1
    g1, g2 = (0.6, c1, z), (0.5, c2, z * (1 + dz_rel))
    _same_branches(_branches(r, 8, 8), [_composite([g1, g2], C_BG), _composite([g2, g1], C_BG)])
    # the FP64 order (nearer first) is the primary branch
    np.testing.assert_allclose(r.rgb[8, 8], _composite([g1, g2], C_BG)[:3], atol=1e-12)


def test_separated_pair_is_not_an_order_tie():
    sc = _two_on_axis(1e-3)                       # 4 mm apart: far outside the bands
    r = O.render_view(sc, 0, 0, opts(bg=tuple(C_BG)))
    assert r.ambiguous_by_kind["order"] == 0 and r.n_alt[8, 8] == 0


def test_order_tie_with_a_skipped_gaussian_is_not_ambiguous():
    # the second Gaussian's alpha (1e-3) is far below alpha_min: it is skipped in either order
    sc = _two_on_axis(2.5e-8, alphas=(0.6, 1e-3))
    r = O.render_view(sc, 0, 0, opts(bg=tuple(C_BG)))
    assert r.ambiguous_by_kind["order"] == 0 and r.n_alt[8, 8] == 0


def test_three_way_depth_tie_returns_every_order():
    import itertools
    z = 3.0
    cols = [C_FG, np.array([0.1, 0.8, 0.5]), np.array([0.6, 0.6, 0.0])]
    alphas = [0.6, 0.5, 0.4]
    nd = U.node([[0, 0, z]] * 3, log_scales=np.full((3, 3), math.log(0.08)),
                logits=[math.log(a / (1 - a)) for a in alphas], sh=U.colour_sh(np.asarray(cols)), dtype=np.float64)
    sc = U.single_view([nd], f=100.0, W=17, H=17, cx=8.5, cy=8.5)
    r = O.render_view(sc, 0, 0, opts(bg=tuple(C_BG)))
    g = [(alphas[i], cols[i], z) for i in range(3)]
    want = [_composite([g[i] for i in perm], C_BG) for perm in itertools.permutations(range(3))]
    assert r.n_alt[8, 8] == 5
    _same_branches(_branches(r, 8, 8), want)
    # exact ties in FP64 take the id order on the primary branch
    np.testing.assert_allclose(r.rgb[8, 8], want[0][:3], atol=1e-12)


def test_branch_budget_widens_over_every_order():
    # with no flips allowed the tolerance must cover the other order
    sc = _two_on_axis(2.5e-8)
    r = O.render_view(sc, 0, 0, opts(bg=tuple(C_BG), max_flips=0))
    assert r.n_alt[8, 8] == 0 and r.widened_pixels >= 1
    g1, g2 = (0.6, C_FG, 4.0), (0.5, np.array([0.1, 0.8, 0.5]), 4.0 * (1 + 2.5e-8))
    other = _composite([g2, g1], C_BG)
    here = np.r_[r.rgb[8, 8], r.depth[8, 8]]
    assert r.tol_rgb[8, 8] >= np.abs(other[:3] - here[:3]).max() - 1e-15
    assert r.tol_d[8, 8] >= abs(other[3] - here[3]) - 1e-15


def test_centre_on_the_near_plane_returns_culled_and_kept_branches():
    zn, p = 0.01, 0.4
    # f sigma / z = 1 px at the near plane; the centre projects onto the centre of pixel (8, 8)
    nd = U.node([[0, 0, zn]], log_scales=np.full((1, 3), math.log(1e-4)), logits=[math.log(p / (1 - p))],
                sh=U.colour_sh([C_FG]), dtype=np.float64)
    sc = U.single_view([nd], f=100.0, W=17, H=17, cx=8.5, cy=8.5)
    r = O.render_view(sc, 0, 0, opts(z_near=zn, bg=tuple(C_BG)))
    assert r.ambiguous_by_kind["near"] >= 1 and r.n_alt[8, 8] == 1
    _same_branches(_branches(r, 8, 8), [np.r_[p * C_FG + (1 - p) * C_BG, p * zn, p], np.r_[C_BG, 0, 0]])
    # a centre well in front of the plane is kept with no alternative
    r2 = O.render_view(sc, 0, 0, opts(z_near=zn * 0.9, bg=tuple(C_BG)))
    assert r2.ambiguous_by_kind["near"] == 0 and r2.n_alt[8, 8] == 0 and r2.alpha[8, 8] == pytest.approx(p, rel=1e-12)


def test_coverage_error_bound_grows_with_the_composited_gaussians():
    # the FP32 error bound of the coverage is zero on an empty pixel, positive where Gaussians are
    # composited, and every branch carries its own
    sc = _two_on_axis(2.5e-8)
    r = O.render_view(sc, 0, 0, opts(bg=tuple(C_BG)))
    assert r.err_a[0, 0] == 0.0 and r.alpha[0, 0] == 0.0
    assert 0 < r.err_a[8, 8] < 1e-4
    assert np.all(r.alternatives(8 * 17 + 8)[:, 5] > 0)
