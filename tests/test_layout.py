"""dgs_spatial_order (host code, no GPU): a permutation along a Z-order curve of the means."""
import numpy as np
import pytest

from paper_2507_21981_gb300 import build as B
from paper_2507_21981_gb300 import dgs as D
from paper_2507_21981_gb300 import scenes as S


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    return D.load()


def _morton(mean):
    """Independent restatement: 21-bit cells of one size over the bounding box, bit i of the
    x/y/z cell index at bit 3i/3i+1/3i+2 of the code."""
    m = mean.astype(np.float64)
    lo, hi = m.min(0), m.max(0)
    ext = (hi - lo).max()
    q = np.clip(np.floor((m - lo) * ((2 ** 21 - 1) / ext)), 0, 2 ** 21 - 1).astype(np.uint64)
    code = np.zeros(len(m), np.uint64)
    for bit in range(21):
        for a in range(3):
            code |= ((q[:, a] >> np.uint64(bit)) & np.uint64(1)) << np.uint64(3 * bit + a)
    return code


def test_is_the_stable_z_order_of_the_means():
    rng = np.random.default_rng(0)
    mean = rng.normal(size=(5000, 3)).astype(np.float32)
    mean[100] = mean[7]                                  # a tie: index order
    p = D.dgs_spatial_order(mean)
    assert np.array_equal(np.sort(p), np.arange(len(mean)))
    assert np.array_equal(p, np.lexsort((np.arange(len(mean)), _morton(mean))))


def test_runs_of_32_are_compact_on_the_room():
    room = S.room_node(np.random.default_rng(3), 200_000, sh_degree=0)
    p = D.dgs_spatial_order(room.mean)

    def radius(m):
        c = m.reshape(-1, 32, 3)
        return np.sqrt(((c - c.mean(1, keepdims=True)) ** 2).sum(-1)).max(1)
    n = room.n // 32 * 32
    before, after = np.median(radius(room.mean[:n])), np.median(radius(room.mean[p][:n]))
    assert after < before / 20, (before, after)


def test_edge_cases():
    assert len(D.dgs_spatial_order(np.zeros((0, 3), np.float32))) == 0
    same = np.ones((10, 3), np.float32)                  # zero extent: index order
    assert np.array_equal(D.dgs_spatial_order(same), np.arange(10))
    m = np.random.default_rng(1).normal(size=(50, 3)).astype(np.float32)
    m[[3, 20]] = np.nan
    m[11, 2] = np.inf
    p = D.dgs_spatial_order(m)
    assert list(p[-3:]) == [3, 11, 20]                   # non-finite last, in index order
    lib = D.load()
    assert lib.dgs_spatial_order(None, 5, None) == D.DGS_ERR_INVALID_ARG
    assert lib.dgs_spatial_order(None, -1, None) == D.DGS_ERR_INVALID_ARG
