"""Image randomisation (overlay blend, HSV jitter, gamma) on the GPU against the FP64 oracle.

1. The separate pass (dgs_augment_rgb) on seeded synthetic images, element by element against
   oracle/augment.py.  Tolerance, derived from FP32 arithmetic: the colour before the power
   curve carries at most 2e-6 absolute error (a handful of roundings of values in [0, 6]),
   which the curve c^gamma spreads by gamma_spread(c2, gamma, 2e-6); the power itself,
   2^(gamma log2 c) with the approximate base-2 instructions, adds at most 8e-6 relative.
2. The fused compositor epilogue equals render-then-separate-pass bit for bit (same per-pixel
   function on the same FP32 colour), in eager, graph and plain modes; depth and alpha are
   untouched.
3. The fused render against oracle render + oracle randomisation, per pixel.  The render
   itself matches the oracle within the parity bound e_rgb = 2e-3 + the oracle's own
   tolerance (tests/parity.py); the randomisation before the power curve is Lipschitz in the
   max norm with constant L = max(1, v)(1 + 6 max(1, s)) (blend: 1; value scaling: v; the
   hue term C k(H + h) moves by at most 6 per unit: 2 through the chroma C, 4 through H C),
   so the bound is gamma_spread(c2, gamma, L e_rgb) + the separate pass's own tolerance.
   A check on the CPU shows that this bound still rejects a wrong crop or a wrong step order.
"""
import numpy as np
import pytest

import oracle as O
from oracle import augment as A
from paper_2507_21981_gb300 import scenes as S
from tests.parity import TOL_RGB

torch = pytest.importorskip("torch")


def _gpu_tol(c2, out, gamma):
    return 2e-7 + A.gamma_spread(c2, gamma, 2e-6) + 8e-6 * out


def _lipschitz(p):
    return max(1.0, float(p["val_scale"])) * (1.0 + 6.0 * max(1.0, float(p["sat_scale"])))


def _synthetic_views():
    """Ragged views (1x1 up to larger than the overlay, so crops wrap) of synthetic colour: uniform
    values in [-0.1, 1.2] (the clamp acts) with rows of greys, black, white, primaries and ties."""
    sizes = [(1, 1), (7, 5), (64, 48), (130, 97), (300, 20), (33, 61)]
    rng = np.random.default_rng(21)
    imgs = []
    for (w, h) in sizes:
        x = rng.uniform(-0.1, 1.2, size=(h, w, 3)).astype(np.float32)
        if h >= 4 and w >= 8:
            x[0, :8] = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5], [1, 0, 0], [0, 1, 0], [0, 0, 1],
                                 [0.7, 0.7, 0.2], [0.2, 0.7, 0.7]], np.float32)
            g = rng.uniform(0, 1, size=(w, 1)).astype(np.float32)
            x[1] = np.repeat(g, 3, axis=1)
            x[2, :, 0] = x[2, :, 1]                    # red = green ties
        imgs.append(x)
    return sizes, imgs


def _param_sets(n, ow, oh, n_frames):
    p = S.augment_params(4, n, n_frames, ow, oh, hue=0.5, sat=(0.0, 2.0), val=(0.3, 2.0), gamma=(0.5, 2.0),
                         beta=(0.0, 1.0), p_overlay=0.7)
    p[0]["overlay_beta"] = 1.0
    p[1]["gamma"] = 1.0
    p[1]["overlay_beta"] = 0.0
    p[2]["hue_shift"] = 3.25
    p[3]["sat_scale"] = 0.0
    p[4]["hue_shift"] = -0.7
    return p


@pytest.mark.gpu
def test_separate_pass_matches_oracle_on_synthetic_images():
    from paper_2507_21981_gb300 import dgs as D
    from paper_2507_21981_gb300.render import Renderer
    sizes, imgs = _synthetic_views()
    n_f, ow, oh = 3, 64, 48
    ov = S.overlay_frames(5, n_frames=n_f, width=ow, height=oh)
    prm = _param_sets(len(sizes), ow, oh, n_f)
    # views placed with gaps between them: the gaps must stay untouched
    offs, at = [], 0
    for (w, h) in sizes:
        offs.append(at)
        at += w * h + 17
    buf = np.full((at, 3), np.nan, np.float32)
    for (w, h), x, o in zip(sizes, imgs, offs):
        buf[o:o + w * h] = x.reshape(-1, 3)
    r = Renderer()
    d_ov = torch.as_tensor(ov).cuda()
    r.set_augment(prm, d_ov)
    d_buf = torch.as_tensor(buf).cuda()
    vs = np.asarray(sizes, np.int32)
    rc = D.dgs_augment_rgb(r.ctx, d_buf, vs, np.asarray(offs, np.int64), len(sizes),
                           torch.cuda.current_stream().cuda_stream)
    assert rc == D.DGS_OK, D.dgs_last_error(r.ctx)
    assert r.launches() == 1
    got = d_buf.cpu().numpy()
    torch.cuda.synchronize()
    r.close()
    gaps = np.ones(at, bool)
    for (w, h), o in zip(sizes, offs):
        gaps[o:o + w * h] = False
    assert np.isnan(got[gaps]).all()
    worst = 0.0
    for k, ((w, h), x, o) in enumerate(zip(sizes, imgs, offs)):
        ref, st = A.augment_view(x, prm[k], ov, return_stages=True)
        g = got[o:o + w * h].reshape(h, w, 3).astype(np.float64)
        err = np.abs(g - ref)
        tol = _gpu_tol(st["c2"], ref, float(prm[k]["gamma"]))
        assert (err <= tol).all(), (k, float(err.max()), np.unravel_index(np.argmax(err - tol), err.shape))
        worst = max(worst, float(err.max()))
    assert worst < 1e-3
    # the same views packed back to back (view_pixel_offset = NULL): same results
    packed = np.concatenate([x.reshape(-1, 3) for x in imgs], axis=0)
    r = Renderer()
    r.set_augment(prm, d_ov)
    d_p = torch.as_tensor(packed).cuda()
    assert D.dgs_augment_rgb(r.ctx, d_p, vs, None, len(sizes), torch.cuda.current_stream().cuda_stream) == D.DGS_OK
    gp = d_p.cpu().numpy()
    r.close()
    at = 0
    for (w, h), o in zip(sizes, offs):
        assert np.array_equal(gp[at:at + w * h], got[o:o + w * h])
        at += w * h


def _ragged():
    return S.config3(seed=5, n_envs=7, n_bg=30_000, n_assets=8, asset_lo=500, asset_hi=4_000, max_nodes=4,
                     resolutions=((80, 60), (160, 120), (200, 110)))


def _overlay_dev(n_f=4, w=176, h=144, seed=2):
    ov = S.overlay_frames(seed, n_frames=n_f, width=w, height=h)
    return ov, torch.as_tensor(ov).cuda()


def _host(out):
    return [None if t is None else t.cpu().numpy() for t in out]


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["batched", "graph", "plain"])
def test_fused_epilogue_equals_separate_pass_bitwise(mode):
    from paper_2507_21981_gb300 import dgs as D
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = _ragged()
    ds = DeviceScene(sc, device="cuda:0")
    ov, d_ov = _overlay_dev()
    prm = S.augment_params(9, ds.n_views, ov.shape[0], ov.shape[2], ov.shape[1], p_overlay=0.7)
    base = Renderer(mode="batched")
    rgb0, depth0, alpha0 = base.render(ds)
    base.set_augment(prm, d_ov)
    sep = base.augment_rgb(ds, rgb0.clone())
    want = sep.cpu().numpy()
    r = Renderer(mode=mode)
    r.set_augment(prm, d_ov)
    for _ in range(2 if mode == "graph" else 1):
        got = _host(r.render(ds))
        assert np.array_equal(got[0], want)
        assert np.array_equal(got[1], depth0.cpu().numpy()) and np.array_equal(got[2], alpha0.cpu().numpy())
    if mode == "graph":
        assert r.stats()["path"] == D.DGS_PATH_GRAPH
        # new parameters, same overlay: the replay reads the new records
        prm2 = S.augment_params(10, ds.n_views, ov.shape[0], ov.shape[2], ov.shape[1], p_overlay=0.7)
        r.set_augment(prm2, d_ov)
        got = _host(r.render(ds))
        assert r.stats()["path"] == D.DGS_PATH_GRAPH
        base.set_augment(prm2, d_ov)
        assert np.array_equal(got[0], base.augment_rgb(ds, rgb0.clone()).cpu().numpy())
        # clearing the randomisation recaptures and gives the plain render back
        r.set_augment(None)
        got = _host(r.render(ds))
        assert r.stats()["path"] == D.DGS_PATH_CAPTURED
        assert np.array_equal(got[0], rgb0.cpu().numpy())
    r.close()
    base.close()


def _compare_to_oracle(sc, ds, rgb, prm, ov, views):
    """Fused GPU output of `views` against oracle render + oracle randomisation, per pixel."""
    pk = O.oracle._Packed(sc)
    report = []
    for v in views:
        e, c = sc.views[v]
        ref = O.render_view(sc, e, c, O.OracleOptions(), pk)
        H, W = ref.depth.shape
        p = prm[v]
        want, st = A.augment_view(ref.rgb, p, ov, return_stages=True)
        g = rgb[ds.view_slice(v)].reshape(H, W, 3).astype(np.float64)
        gam = float(p["gamma"])
        e_rgb = _lipschitz(p) * (TOL_RGB + ref.tol_rgb[..., None])
        tol = A.gamma_spread(st["c2"], gam, e_rgb) + _gpu_tol(st["c2"], want, gam)
        err = np.abs(g - want)
        bad = (err > tol).any(axis=-1)
        # pixels whose FP32 decisions may go the other way: any alternative branch will do
        for flat in np.nonzero(bad.reshape(-1))[0]:
            y, x = divmod(int(flat), W)
            q = dict(zip(A.FIELDS, [p[f] for f in A.FIELDS]))
            q["overlay_x"] = (int(p["overlay_x"]) + x) % ov.shape[2]
            q["overlay_y"] = (int(p["overlay_y"]) + y) % ov.shape[1]
            for alt in ref.alternatives(int(flat)):
                a_out, a_st = A.augment_view(np.asarray(alt[:3], np.float64).reshape(1, 1, 3), q, ov, return_stages=True)
                a_tol = A.gamma_spread(a_st["c2"], gam, _lipschitz(p) * (TOL_RGB + ref.tol_rgb[y, x])) + \
                    _gpu_tol(a_st["c2"], a_out, gam)
                if (np.abs(g[y, x] - a_out[0, 0]) <= a_tol[0, 0]).all():
                    bad[y, x] = False
                    break
        report.append(dict(view=v, bad=int(bad.sum()), max_err=float(err.max()),
                           median_err=float(np.median(err)), beta=float(p["overlay_beta"])))
        assert bad.sum() == 0, report[-1]
    return report


@pytest.mark.gpu
def test_fused_render_matches_oracle_render_and_randomisation():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = _ragged()
    ds = DeviceScene(sc, device="cuda:0")
    ov, d_ov = _overlay_dev(seed=3)
    prm = S.augment_params(11, ds.n_views, ov.shape[0], ov.shape[2], ov.shape[1], hue=0.25, sat=(0.7, 1.0),
                           val=(0.7, 1.0), gamma=(0.7, 1.5), beta=(0.3, 0.8), p_overlay=0.8)
    r = Renderer(mode="graph")
    r.set_augment(prm, d_ov)
    rgb = r.render(ds)[0].cpu().numpy()
    r.close()
    rep = _compare_to_oracle(sc, ds, rgb, prm, ov, range(sc.n_views))
    assert max(x["median_err"] for x in rep) < 1e-4


@pytest.mark.gpu
def test_full_batch_fused_randomisation_sampled_views():
    """The benchmark batch (64 envs x 2 cameras 640x480, 1.08M Gaussians per env, Z-ordered) as
    graph replays with the randomisation fused (8-frame 1280x720 overlay clip), as bench.py times
    it; two sampled views against oracle render + oracle randomisation."""
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config2(seed=1)
    ds = DeviceScene(sc, device="cuda:0", spatial_order=True)
    ov = S.overlay_frames(1, n_frames=8, width=1280, height=720)
    prm = S.augment_params(1, ds.n_views, 8, 1280, 720)
    prm[[5, 77]]["overlay_beta"] = 0.35                   # both sampled views blend the overlay
    r = Renderer(mode="graph")
    r.set_augment(prm, torch.as_tensor(ov).cuda())
    for _ in range(2):
        rgb = r.render(ds)[0]
    rgb = rgb.cpu().numpy()
    r.close()
    _compare_to_oracle(ds.scene, ds, rgb, prm, ov, [5, 77])


def test_oracle_bound_rejects_a_wrong_crop_and_a_wrong_order():
    """CPU only: the per-pixel bound used above would catch plausible mistakes.  The mistakes
    are planted in copies of the oracle's own steps on a synthetic image, never on the GPU."""
    rng = np.random.default_rng(3)
    ov = S.overlay_frames(3, n_frames=2, width=176, height=144)
    img = rng.uniform(0, 1, size=(60, 80, 3))
    p = dict(hue_shift=0.1, sat_scale=0.9, val_scale=0.9, gamma=1.2, overlay_beta=0.5, overlay_frame=1,
             overlay_x=40, overlay_y=30)
    want, st = A.augment_view(img, p, ov, return_stages=True)
    tol = A.gamma_spread(st["c2"], 1.2, _lipschitz(p) * TOL_RGB) + _gpu_tol(st["c2"], want, 1.2)
    shifted = dict(p, overlay_x=41)
    bad_crop = A.augment_view(img, shifted, ov)
    assert ((np.abs(bad_crop - want) > tol).any(axis=-1)).mean() > 0.05
    # HSV jitter before the blend instead of after it
    jit = A.augment_view(img, dict(p, overlay_beta=0.0, gamma=1.0), None)
    o = A.overlay_crop(ov, 1, 40, 30, 80, 60)
    wrong = (0.5 * jit + 0.5 * o) ** 1.2
    assert ((np.abs(wrong - want) > tol).any(axis=-1)).mean() > 0.05
