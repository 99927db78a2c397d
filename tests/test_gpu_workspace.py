"""dgs_workspace_query_batch: the device workspace a render of a given batch needs, measured by
its count pass, against what a fresh context holds after rendering that batch."""
import pytest

from paper_2507_21981_gb300 import dgs as D
from paper_2507_21981_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make", [
    lambda: S.config1(seed=1),
    lambda: S.config2(seed=2, n_envs=6, n_bg=60_000, n_obj=2_000, width=160, height=120, f=125.0),
])
def test_query_matches_the_workspace_a_render_takes(make):
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    ds = DeviceScene(make(), device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    q = Renderer(mode="batched")
    rc, need = D.dgs_workspace_query_batch(q.ctx, ds.nodes, ds.n_nodes, ds.env_node_ids, ds.n_envs, ds.max_nodes,
                                           ds.node_poses, ds.cams, ds.cams_per_env, ds.max_cams, None, stream)
    assert rc == D.DGS_OK and need > 0
    # the query allocates the count tables but not the lists
    assert D.dgs_workspace_query(q.ctx) < need
    q.close()
    r = Renderer(mode="batched")
    r.render(ds)
    torch.cuda.synchronize()
    held = D.dgs_workspace_query(r.ctx)
    # every allocation keeps 25 % growth slack (and at least 256 bytes)
    assert need <= held <= 1.25 * need + 64 * 256, (need, held)
    r.close()


def test_query_validates_like_render():
    from paper_2507_21981_gb300.render import Renderer
    r = Renderer()
    rc, _ = D.dgs_workspace_query_batch(r.ctx, None, 0, None, 1, 1, None, None, None, 1, None,
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == D.DGS_ERR_INVALID_ARG
    r.close()
