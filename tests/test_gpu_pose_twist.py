"""se(3) twist of pose gradients (dgs_pose_twist_grad through the C ABI) against the oracle's
FP64 restatement, on random rigid poses and on the pose gradients of a rendered view."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2507_21981_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rigid_poses(rng, n):
    R = Rotation.random(n, random_state=rng).as_matrix()
    t = rng.normal(size=(n, 3)) * 2.0
    return np.concatenate([R, t[:, :, None]], axis=2).astype(np.float32)


def _twist_gpu(P, G):
    from paper_2507_21981_gb300.render import pose_twist_grad
    out = pose_twist_grad(torch.from_numpy(P).cuda(), torch.from_numpy(G).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def test_twist_matches_oracle_on_random_poses():
    rng = np.random.default_rng(0)
    for n in (1, 7, 1000):
        P = _rigid_poses(rng, n)
        G = rng.normal(size=(n, 3, 4)).astype(np.float32)
        got = _twist_gpu(P, G)
        want = np.stack([O.pose_twist_grad(P[i].astype(np.float64), G[i].astype(np.float64)) for i in range(n)])
        assert got.shape == (n, 6)
        # FP32: a 3-term dot product of magnitude <= |G| |T| per entry, then one difference
        scale = np.abs(G).max(axis=(1, 2)) * (1 + np.abs(P).max(axis=(1, 2)))
        assert np.all(np.abs(got - want) <= 1e-6 * scale[:, None] * 8)


def test_twist_of_rendered_pose_gradients():
    """The twist of the GPU's 3x4 pose gradients equals the oracle's twist of its own pose
    gradients within the pose-gradient tolerance carried through the twist map."""
    from paper_2507_21981_gb300.render import DeviceScene, Renderer
    sc = S.config1(seed=3)
    ds = DeviceScene(sc, device="cuda:0")
    r = Renderer()
    rgb, depth, _ = r.render(ds)
    rng = np.random.default_rng(1)
    ref = O.render_view(sc, 0, 0)
    amb = (ref.n_alt > 0) | (ref.tol_rgb > 0) | ref.grad_amb
    g = rng.normal(size=ref.rgb.shape).astype(np.float32)
    g[amb] = 0
    _, gposes = r.backward(ds, rgb, depth, torch.from_numpy(g.reshape(-1, 3)).cuda(), None)
    torch.cuda.synchronize()
    r.close()
    poses = ds.node_poses.reshape(-1, 3, 4)
    from paper_2507_21981_gb300.render import pose_twist_grad
    tw = pose_twist_grad(poses, gposes.reshape(-1, 3, 4)).cpu().numpy().astype(np.float64)
    gref = O.backward_view(sc, 0, 0, g.astype(np.float64))["pose"].reshape(-1, 3, 4)
    P64 = poses.cpu().numpy().astype(np.float64)
    want = np.stack([O.pose_twist_grad(P64[i], gref[i]) for i in range(len(P64))])
    present = sc.env_node_ids.reshape(-1) >= 0
    scale = np.abs(want[present]).max()
    assert np.abs(tw[present] - want[present]).max() <= 1e-3 * scale
