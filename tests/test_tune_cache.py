"""The autotuner's cache (render.TuneCache): its key classes batches by GPU name, view
resolutions, view count and Gaussians per view (both rounded to powers of two), and its JSON
file round-trips what autotune stores.  Needs no GPU: DeviceScene tables on the CPU."""
import json

import pytest

torch = pytest.importorskip("torch")

from paper_2507_21981_gb300 import scenes as S
from paper_2507_21981_gb300.render import DeviceScene, TuneCache


def _ds(**kw):
    return DeviceScene(S.config2(**kw), device="cpu")


def test_key_classes_batches():
    a = TuneCache.key(_ds(seed=1, n_envs=4, n_bg=20_000, n_obj=500, width=160, height=120), "GPU")
    b = TuneCache.key(_ds(seed=2, n_envs=4, n_bg=21_000, n_obj=500, width=160, height=120), "GPU")
    assert a == b                                                         # same class
    c = TuneCache.key(_ds(seed=1, n_envs=4, n_bg=20_000, n_obj=500, width=320, height=240), "GPU")
    d = TuneCache.key(_ds(seed=1, n_envs=16, n_bg=20_000, n_obj=500, width=160, height=120), "GPU")
    e = TuneCache.key(_ds(seed=1, n_envs=4, n_bg=90_000, n_obj=500, width=160, height=120), "GPU")
    f = TuneCache.key(_ds(seed=1, n_envs=4, n_bg=20_000, n_obj=500, width=160, height=120), "other GPU")
    assert len({a, c, d, e, f}) == 5                                      # resolution, views, density, GPU


def test_store_and_load_round_trip(tmp_path):
    path = tmp_path / "tune.json"
    c = TuneCache(str(path))
    assert c.get("k") is None
    c.put("k", (32, 8), {(16, 16): 1.5, (32, 8): 1.25})
    c.put("k2", (8, 8), {(8, 8): 2.0})
    assert c.get("k") == ((32, 8), {(16, 16): 1.5, (32, 8): 1.25})
    assert TuneCache(str(path)).get("k2") == ((8, 8), {(8, 8): 2.0})
    data = json.loads(path.read_text())
    assert data["k"]["best"] == [32, 8] and set(data) == {"k", "k2"}
