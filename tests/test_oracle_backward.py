"""Pins of the oracle's analytic adjoint: FP64 central finite differences of the oracle's
forward pass, a closed form for the degree-0 SH gradient, and the se(3) twist gradient."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import oracle as O
from paper_2507_21981_gb300 import scenes as S
from tests import scene_utils as U

OPTS = O.OracleOptions(nthreads=4)


def _f64(sc, sh_degree=None, seed=0):
    """Copy of a scene with float64 arrays (optionally with random SH of a higher degree)."""
    rng = np.random.default_rng(seed)
    nodes = []
    for nd in sc.nodes:
        deg = nd.sh_degree if sh_degree is None else sh_degree
        sh = nd.sh.astype(np.float64)
        if deg != nd.sh_degree:
            extra = rng.normal(0, 0.2, (nd.n, (deg + 1) ** 2, 3))
            extra[:, 0] = sh[:, 0]
            sh = extra
        nodes.append(S.GaussianNode(nd.mean.astype(np.float64), nd.log_scale.astype(np.float64),
                                    nd.quat.astype(np.float64), nd.opacity_logit.astype(np.float64), sh, deg))
    return S.Scene(sc.name, nodes, sc.env_node_ids, sc.node_poses.astype(np.float64), sc.cams_per_env,
                   sc.cam_intr.astype(np.float64), sc.cam_res, sc.cam_pose.astype(np.float64))


def _loss(sc, gC, gD):
    r = O.render_view(sc, 0, 0, OPTS)
    return float((gC * r.rgb).sum() + (gD * r.depth).sum()), r.decision_hash


def _fd_check(sc, n_per_group=40, seed=0, rtol=2e-5):
    rng = np.random.default_rng(seed)
    W, H = (int(x) for x in sc.cam_res[0, 0])
    gC = rng.normal(size=(H, W, 3))
    gD = rng.normal(size=(H, W)) * 0.3
    g = O.backward_view(sc, 0, 0, gC, gD, OPTS)
    _, h0 = _loss(sc, gC, gD)
    offs = np.concatenate([[0], np.cumsum([nd.n for nd in sc.nodes])])
    checked = excluded = 0
    groups = [("mean", 3), ("log_scale", 3), ("quat", 4), ("opacity_logit", 1), ("sh", None)]
    for name, width in groups:
        G = g[name]
        scale = np.abs(G).max()
        for _ in range(n_per_group):
            k = int(rng.integers(len(sc.nodes)))
            i = int(rng.integers(sc.nodes[k].n))
            arr = getattr(sc.nodes[k], name)
            if name == "sh":
                idx = (i, int(rng.integers(arr.shape[1])), int(rng.integers(3)))
                analytic = G[offs[k] + i, idx[1], idx[2]]
            elif width == 1:
                idx = (i,)
                analytic = G[offs[k] + i]
            else:
                j = int(rng.integers(width))
                idx = (i, j)
                analytic = G[offs[k] + i, j]
            x0 = arr[idx]
            h = 1e-6 * max(1.0, abs(x0))
            arr[idx] = x0 + h
            lp, hp = _loss(sc, gC, gD)
            arr[idx] = x0 - h
            lm, hm = _loss(sc, gC, gD)
            arr[idx] = x0
            if hp != h0 or hm != h0:
                excluded += 1
                continue
            fd = (lp - lm) / (2 * h)
            assert abs(analytic - fd) <= rtol * abs(fd) + 1e-7 * scale + 1e-9, (name, k, idx, analytic, fd)
            checked += 1
    # node poses (3x4 entries)
    Gp = g["pose"]
    for j in range(sc.env_node_ids.shape[1]):
        for a in range(3):
            for b in range(4):
                x0 = sc.node_poses[0, j, a, b]
                h = 1e-6
                sc.node_poses[0, j, a, b] = x0 + h
                lp, hp = _loss(sc, gC, gD)
                sc.node_poses[0, j, a, b] = x0 - h
                lm, hm = _loss(sc, gC, gD)
                sc.node_poses[0, j, a, b] = x0
                if hp != h0 or hm != h0:
                    excluded += 1
                    continue
                fd = (lp - lm) / (2 * h)
                assert abs(Gp[0, j, a, b] - fd) <= rtol * abs(fd) + 1e-7 * np.abs(Gp).max() + 1e-9, ("pose", j, a, b, Gp[0, j, a, b], fd)
                checked += 1
    return checked, excluded


def test_backward_matches_fd_degree0():
    checked, excluded = _fd_check(_f64(S.fd_subset(seed=1)), seed=1)
    assert checked >= 150 and excluded <= checked // 5


def test_backward_matches_fd_degree3_posed():
    sc = _f64(S.fd_subset(seed=2), sh_degree=3, seed=2)
    checked, excluded = _fd_check(sc, seed=2)
    assert checked >= 150 and excluded <= checked // 5


def test_backward_matches_fd_with_background_and_clamped_jacobian():
    """Wide-angle view: several Gaussians sit beyond the Jacobian guard; coloured background."""
    sc = _f64(S.fd_subset(seed=3), sh_degree=1, seed=3)
    sc.cam_intr[0, 0, :2] = 10.0        # f = 10 on 32 px: half-FOV tangent 1.6
    global OPTS
    saved = OPTS
    OPTS = O.OracleOptions(nthreads=4, bg=(0.3, 0.1, 0.7))
    try:
        checked, excluded = _fd_check(sc, seed=3)
    finally:
        OPTS = saved
    assert checked >= 150 and excluded <= checked // 5


def test_sh00_gradient_closed_form():
    """For one Gaussian with an unclamped colour, dL/dsh_00[ch] = Y00 * sum_p alpha_p gC[p,ch]."""
    nd = U.node([[0.05, -0.03, 3.0]], log_scales=np.full((1, 3), math.log(0.1)), logits=[0.5],
                sh=U.colour_sh([[0.4, 0.5, 0.6]]), dtype=np.float64)
    sc = U.single_view([nd], f=40.0)
    rng = np.random.default_rng(5)
    gC = rng.normal(size=(32, 32, 3))
    r = O.render_view(sc, 0, 0, OPTS)
    g = O.backward_view(sc, 0, 0, gC, np.zeros((32, 32)), OPTS)
    want = U.Y00 * (r.alpha[..., None] * gC).sum(axis=(0, 1))
    np.testing.assert_allclose(g["sh"][0, 0], want, rtol=1e-12)


def _hat(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


def test_pose_twist_gradient_matches_fd():
    sc = _f64(S.fd_subset(seed=6), sh_degree=2, seed=6)
    rng = np.random.default_rng(6)
    gC = rng.normal(size=(32, 32, 3))
    gD = rng.normal(size=(32, 32)) * 0.3
    g = O.backward_view(sc, 0, 0, gC, gD, OPTS)
    P0 = sc.node_poses[0, 1].copy()
    tw = O.pose_twist_grad(P0, g["pose"][0, 1])
    _, h0 = _loss(sc, gC, gD)
    for k in range(6):
        h = 1e-6
        vals = []
        for s in (+1, -1):
            xi = np.zeros(6); xi[k] = s * h
            T = np.zeros((4, 4))
            T[:3, :3] = _hat(xi[3:]); T[:3, 3] = xi[:3]
            E = expm(T)                  # exp of the se(3) element [[phi^, rho], [0, 0]]
            M = np.eye(4); M[:3] = P0
            sc.node_poses[0, 1] = (E @ M)[:3]
            l, hh = _loss(sc, gC, gD)
            assert hh == h0
            vals.append(l)
        sc.node_poses[0, 1] = P0
        fd = (vals[0] - vals[1]) / (2 * h)
        assert tw[k] == pytest.approx(fd, rel=2e-5, abs=1e-7 * np.abs(tw).max())


# --------------------------------------------------------------------------- FP32 error model of the adjoint
def _err_case():
    sc = S.fd_subset(seed=4)
    nd = sc.nodes[0].subset(slice(0, sc.nodes[0].n))
    nd.mean = nd.mean.copy()
    nd.mean[0] = (100.0, 100.0, 5.0)           # far outside the image: composited nowhere
    sc.nodes = [nd] + list(sc.nodes[1:])
    g = np.random.default_rng(3).normal(size=(32, 32, 3))
    return sc, g


def test_gradient_error_model_is_nonnegative_and_vanishes_without_contributions():
    sc, g = _err_case()
    out = O.backward_view(sc, 0, 0, g, with_error=True)
    for name in ("mean", "log_scale", "quat", "opacity_logit", "sh", "pose"):
        e = out["err_" + name]
        assert np.all(np.isfinite(e)) and np.all(e >= 0), name
    # Gaussians whose gradient is exactly zero (composited nowhere) carry no error either
    none = np.all(out["mean"] == 0, axis=1) & (out["opacity_logit"] == 0)
    assert none.any() and np.all(out["err_mean"][none] == 0) and np.all(out["err_opacity_logit"][none] == 0)
    some = ~none
    assert np.all(out["err_opacity_logit"][some] > 0)


def test_gradient_error_model_is_linear_in_the_upstream_gradient():
    sc, g = _err_case()
    a = O.backward_view(sc, 0, 0, g, with_error=True)
    b = O.backward_view(sc, 0, 0, 2.0 * g, with_error=True)
    for name in ("mean", "quat", "sh", "pose"):
        np.testing.assert_allclose(b["err_" + name], 2.0 * a["err_" + name], rtol=1e-12, atol=1e-300)


def test_gradient_error_model_flags_a_cancelling_entry():
    """A round Gaussian centred on a pixel corner under a colour gradient symmetric about it:
    dL/dmean_x is a sum of per-pixel terms of both signs that cancel exactly, so the FP32 model
    must exceed the (vanishing) value itself, while it stays far below the terms' magnitude."""
    nd = U.node([[0.0, 0.0, 4.0]], log_scales=np.full((1, 3), math.log(0.12)), logits=[2.0],
                sh=U.colour_sh([[0.8, 0.4, 0.2]]), dtype=np.float64)
    sc = U.single_view([nd], f=100.0, W=16, H=16, cx=8.0, cy=8.0)
    g = np.ones((16, 16, 3))
    out = O.backward_view(sc, 0, 0, g, with_error=True)
    gx, ex = out["mean"][0, 0], out["err_mean"][0, 0]
    assert abs(gx) < 1e-9 and ex > 10 * abs(gx)
    # the per-pixel terms: the mean's gradient when only the pixels left of the centre are weighted
    gl = g.copy()
    gl[:, 8:] = 0
    half = abs(O.backward_view(sc, 0, 0, gl)["mean"][0, 0])
    assert half > 0 and ex < 1e-4 * half
