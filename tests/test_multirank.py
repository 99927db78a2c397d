"""The multi-GPU form of the benchmark on CPU: two gloo ranks.  Every (env, camera) view is
independent, so ranks render disjoint env batches (weak scaling) and the only collective is
the max of the ranks' times."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        assert bench._dist() == (rank, world, rank)
        ms = bench.max_over_ranks(10.0 + 3.0 * rank, world, "cpu")
        sc = bench.rank_scene(rank, envs=3, n_bg=2_000, n_obj=200, width=64, height=48, f=50.0)
        q.put((rank, ms, sc.n_views, sc.n_pixels, sc.node_poses.copy(), sc.cam_pose.copy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_nothing_but_the_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        r, ms, nv, npx, poses, cams = q.get(timeout=120)
        got[r] = (ms, nv, npx, poses, cams)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time
    assert got[0][0] == got[1][0] == 13.0
    # weak scaling: the same amount of work per rank, different environments
    assert got[0][1] == got[1][1] == 6 and got[0][2] == got[1][2]
    assert not np.allclose(got[0][3], got[1][3]) and not np.allclose(got[0][4], got[1][4])


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(4.5, 1) == 4.5
