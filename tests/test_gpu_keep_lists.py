"""dgs_options.keep_lists: the backward differentiates the lists its forward kept.

With the option, an eager render leaves its view groups' lists on the context, and
dgs_render_backward of the same batch skips staging, counting and binning (stats.path =
DGS_PATH_KEPT_LISTS).  The lists are the ones the backward would have built, so the gradients
must equal those of the rebuilding backward up to the summation order of the adjoint's atomics,
and stay within the oracle's bound.  Any other batch, a render of another batch in between, or
new options must make the backward bin again.
"""
import numpy as np
import pytest

from paper_2507_21981_gb300 import dgs as D
from paper_2507_21981_gb300 import scenes as S
from tests.test_gpu_backward import _compare, _gradients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _grads(r, ds, rgb, depth, seed=0):
    gen = torch.Generator(device="cuda").manual_seed(seed)
    gC = torch.randn(rgb.shape, device="cuda", generator=gen)
    gD = torch.randn(depth.shape, device="cuda", generator=gen)
    ng, gp = r.backward(ds, rgb, depth, gC, gD)
    torch.cuda.synchronize()
    return [{k: v.cpu().numpy() for k, v in g.items()} for g in ng] + [gp.cpu().numpy()], r.stats()["path"]


def _close(a, b):
    for x, y in zip(a[:-1], b[:-1]):
        for k in x:
            np.testing.assert_allclose(y[k], x[k], rtol=1e-4, atol=1e-6 * max(np.abs(x[k]).max(), 1e-30), err_msg=k)
    np.testing.assert_allclose(b[-1], a[-1], rtol=1e-4, atol=1e-6 * np.abs(a[-1]).max())


@pytest.mark.parametrize("views_per_group", [0, 2])
def test_kept_lists_give_the_rebuilt_gradients(views_per_group):
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    # 2 envs x 2 cameras: one view group, or two groups of two views (both kept)
    sc = S.config2(seed=7, n_envs=2, n_bg=30_000, n_obj=1_000, width=160, height=120, f=125.0)
    ds = DeviceScene(sc, device="cuda:0")
    ref_r = Renderer(mode="batched", views_per_group=views_per_group)
    rgb, depth, _ = ref_r.render(ds)
    ref, path = _grads(ref_r, ds, rgb, depth)
    assert path == D.DGS_PATH_EAGER
    r = Renderer(mode="batched", views_per_group=views_per_group, keep_lists=1)
    rgb2, depth2, _ = r.render(ds)
    assert torch.equal(rgb, rgb2) and torch.equal(depth, depth2)
    got, path = _grads(r, ds, rgb2, depth2)
    assert path == D.DGS_PATH_KEPT_LISTS
    _close(ref, got)
    # a second backward of the same forward still finds the lists
    got2, path = _grads(r, ds, rgb2, depth2, seed=0)
    assert path == D.DGS_PATH_KEPT_LISTS
    _close(ref, got2)
    ref_r.close()
    r.close()


def test_graph_replay_keeps_its_lists():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config2(seed=7, n_envs=2, n_bg=30_000, n_obj=1_000, width=160, height=120, f=125.0)
    ds = DeviceScene(sc, device="cuda:0")
    ref_r = Renderer(mode="batched")
    rgb, depth, _ = ref_r.render(ds)
    ref, _ = _grads(ref_r, ds, rgb, depth)
    for vpg in (0, 2):
        r = Renderer(mode="graph", keep_lists=1, views_per_group=vpg)
        r.render(ds)                                   # renders eagerly and captures
        rgb2, depth2, _ = r.render(ds)                 # replays
        assert r.stats()["path"] == D.DGS_PATH_GRAPH
        assert torch.equal(rgb, rgb2) and torch.equal(depth, depth2)
        got, path = _grads(r, ds, rgb2, depth2)
        assert path == D.DGS_PATH_KEPT_LISTS
        _close(ref, got)
        r.close()
    ref_r.close()


def test_another_batch_or_new_options_make_the_backward_bin_again():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sa = S.config2(seed=7, n_envs=2, n_bg=30_000, n_obj=1_000, width=160, height=120, f=125.0)
    sb = S.config2(seed=8, n_envs=1, n_bg=20_000, n_obj=1_000, width=96, height=64, f=75.0)
    da, db = DeviceScene(sa, device="cuda:0"), DeviceScene(sb, device="cuda:0")
    ref_r = Renderer(mode="batched")
    rgb, depth, _ = ref_r.render(da)
    ref, _ = _grads(ref_r, da, rgb, depth)
    r = Renderer(mode="batched", keep_lists=1)
    rgb, depth, _ = r.render(da)
    r.render(db)                                   # another batch replaces the kept lists
    got, path = _grads(r, da, rgb, depth)
    assert path == D.DGS_PATH_EAGER
    _close(ref, got)
    rgb, depth, _ = r.render(da)
    r.set_options(keep_lists=1)                    # new options drop them
    got, path = _grads(r, da, rgb, depth)
    assert path == D.DGS_PATH_EAGER
    _close(ref, got)
    rgb, depth, _ = r.render(da)
    da.cams[0].fx *= 1.001                         # other cameras: another batch
    got, path = _grads(r, da, rgb, depth)
    assert path == D.DGS_PATH_EAGER
    da.cams[0].fx /= 1.001
    ref_r.close()
    r.close()


def test_three_view_groups_are_not_kept():
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config2(seed=7, n_envs=3, n_bg=20_000, n_obj=1_000, width=96, height=64, f=75.0)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer(mode="batched", views_per_group=2, keep_lists=1)
    rgb, depth, _ = r.render(ds)
    assert r.stats()["n_groups"] == 3
    _, path = _grads(r, ds, rgb, depth)
    assert path == D.DGS_PATH_EAGER
    r.close()


def test_kept_lists_backward_against_the_oracle():
    sc = S.config4(seed=2, n_bg=30_000, n_obj=2_000, res=160, f=140.0)
    _compare(sc, *_gradients(sc, seed=4, keep_lists=1))


def test_gradient_buffers_made_once_give_the_fresh_gradients():
    from paper_2507_21981_gb300.render import DeviceScene, GradBuffers, Renderer
    sc = S.config2(seed=7, n_envs=2, n_bg=30_000, n_obj=1_000, width=160, height=120, f=125.0)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer(mode="batched", keep_lists=1)
    rgb, depth, _ = r.render(ds)
    ref, _ = _grads(r, ds, rgb, depth)
    gb = GradBuffers(ds)
    gen = torch.Generator(device="cuda").manual_seed(0)
    gC = torch.randn(rgb.shape, device="cuda", generator=gen)
    gD = torch.randn(depth.shape, device="cuda", generator=gen)
    for _ in range(2):                      # the second call must start from zero again
        ng, gp = r.backward(ds, rgb, depth, gC, gD, out=gb)
        torch.cuda.synchronize()
        got = [{k: v.cpu().numpy() for k, v in g.items()} for g in ng] + [gp.cpu().numpy()]
        _close(ref, got)
    assert ng is gb.node_grads
    r.close()


@pytest.mark.parametrize("mode", ["batched", "graph"])
def test_long_lists_replay_in_checkpointed_segments(mode):
    """A dense view whose tile lists run to thousands of entries: the kept-lists adjoint replays
    512-entry segments in parallel from the forward's checkpoints and must give the gradients of
    the sequential replay (the default backward, which bins again)."""
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config4(seed=3, n_bg=120_000, n_obj=4_000, res=128, f=110.0)
    ds = DeviceScene(sc, device="cuda:0")
    ref_r = Renderer(mode="batched")
    rgb, depth, _ = ref_r.render(ds)
    st = ref_r.stats()
    assert st["n_pairs"] / (128 * 128 / 256) > 2 * 512      # lists of several segments on average
    ref, path = _grads(ref_r, ds, rgb, depth)
    assert path == D.DGS_PATH_EAGER
    r = Renderer(mode=mode, keep_lists=1)
    for _ in range(2 if mode == "graph" else 1):
        rgb2, depth2, _ = r.render(ds)
    assert torch.equal(rgb, rgb2) and torch.equal(depth, depth2)
    got, path = _grads(r, ds, rgb2, depth2)
    assert path == D.DGS_PATH_KEPT_LISTS
    _close(ref, got)
    ref_r.close()
    r.close()
