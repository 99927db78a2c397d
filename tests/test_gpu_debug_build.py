"""The bounds-checked build (libdgs_debug.so, compiled with -DDGS_DEBUG).

Its kernels check every index they take from another kernel's output before the access.  On
correct inputs no check may fire, and the images must be bit-identical to the release build's
(the checks only guard accesses).  dgs_options.test_fault = 3 tells the compositors that each
view group holds half the records it does: the check on tile-list entries must then end the
call with DGS_ERR_CUDA naming that check, in the forward and in the adjoint, and the context must
render correctly afterwards.  Every access the shortened bound lets through lies inside the
records written, so the planted failure cannot reach memory it should not.
"""
import numpy as np
import pytest

from paper_2507_21981_gb300 import build as B
from paper_2507_21981_gb300 import dgs as D
from paper_2507_21981_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    lib = D.load(B.build(debug=True))
    assert lib.dgs_build_flags() == D.DGS_BUILD_DEBUG
    return lib


def _scene():
    return S.config2(seed=5, n_envs=3, n_bg=40_000, n_obj=1_500, width=160, height=120, f=125.0)


def _render(lib, sc, mode, renders=1, **opts):
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    with D.using(lib):
        ds = DeviceScene(sc, device="cuda:0")
        r = Renderer(mode=mode, **opts)
        for _ in range(renders):
            out = [t.cpu().numpy() for t in r.render(ds)]
        torch.cuda.synchronize()
        r.close()
    return out


@pytest.mark.parametrize("mode,renders", [("batched", 1), ("plain", 1), ("graph", 2)])
def test_debug_build_renders_bit_identically(dbg, mode, renders):
    sc = _scene()
    ref = _render(D.load(), sc, mode, renders)
    got = _render(dbg, sc, mode, renders)
    for a, b, name in zip(ref, got, ("rgb", "depth", "alpha")):
        assert np.array_equal(a, b), (mode, name, float(np.abs(a - b).max()))


def test_debug_build_backward_passes_its_checks(dbg):
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config4(seed=2, n_bg=30_000, n_obj=2_000, res=160, f=140.0)
    grads = []
    for lib in (D.load(), dbg):
        with D.using(lib):
            ds = DeviceScene(sc, device="cuda:0")
            r = Renderer(mode="batched")
            rgb, depth, _ = r.render(ds)
            gen = torch.Generator(device="cuda").manual_seed(0)
            gC = torch.randn(rgb.shape, device="cuda", generator=gen)
            gD = torch.randn(depth.shape, device="cuda", generator=gen)
            node_grads, gposes = r.backward(ds, rgb, depth, gC, gD)
            torch.cuda.synchronize()
            grads.append([{k: v.cpu().numpy() for k, v in g.items()} for g in node_grads] + [gposes.cpu().numpy()])
            r.close()
    # the adjoint accumulates with atomics, so the two runs may differ in summation order only
    for a, b in zip(grads[0][:-1], grads[1][:-1]):
        for k in a:
            np.testing.assert_allclose(b[k], a[k], rtol=1e-4, atol=1e-6 * max(np.abs(a[k]).max(), 1e-30))
    np.testing.assert_allclose(grads[1][-1], grads[0][-1], rtol=1e-4, atol=1e-6 * np.abs(grads[0][-1]).max())


def test_short_record_bound_is_reported_by_the_forward_and_the_adjoint(dbg):
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = _scene()
    ref = _render(D.load(), sc, "batched")
    with D.using(dbg):
        ds = DeviceScene(sc, device="cuda:0")
        r = Renderer(mode="batched")
        rgb, depth, _ = r.render(ds)
        gC = torch.ones_like(rgb)
        gD = torch.ones_like(depth)
        r.set_options(test_fault=3)
        with pytest.raises(D.DgsError) as ei:
            r.render(ds)
        assert ei.value.code == D.DGS_ERR_CUDA
        assert "debug bounds check failed (compositor: instance number" in str(ei.value), str(ei.value)
        with pytest.raises(D.DgsError) as ei:
            r.backward(ds, rgb, depth, gC, gD)
        assert ei.value.code == D.DGS_ERR_CUDA
        assert "adjoint compositor: instance number" in str(ei.value), str(ei.value)
        r.set_options(test_fault=0)
        out = [t.cpu().numpy() for t in r.render(ds)]
        torch.cuda.synchronize()
        r.close()
    for a, b in zip(ref, out):
        assert np.array_equal(a, b)
