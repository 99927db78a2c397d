"""Small hand-built scenes for closed-form checks (inputs only, no renderer arithmetic)."""
import math

import numpy as np

from paper_2507_21981_gb300 import scenes as S

Y00 = 0.5 / math.sqrt(math.pi)
IDENT = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)


def node(means, log_scales=None, quats=None, logits=None, sh=None, deg=0, dtype=np.float32):
    means = np.asarray(means, np.float64).reshape(-1, 3)
    n = means.shape[0]
    if log_scales is None:
        log_scales = np.full((n, 3), math.log(0.05))
    if quats is None:
        quats = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    if logits is None:
        logits = np.zeros(n)
    ncoef = (deg + 1) ** 2
    if sh is None:
        sh = np.zeros((n, ncoef, 3))
    arr = lambda a, shape: np.ascontiguousarray(np.asarray(a, np.float64).reshape(shape).astype(dtype))
    return S.GaussianNode(arr(means, (n, 3)), arr(log_scales, (n, 3)), arr(quats, (n, 4)), arr(logits, (n,)),
                          arr(sh, (n, ncoef, 3)), deg)


def colour_sh(rgb):
    """Degree-0 coefficients giving colour rgb (before the max(0, .) clamp)."""
    return ((np.asarray(rgb, np.float64) - 0.5) / Y00).reshape(-1, 1, 3)


def single_view(nodes, poses=None, f=50.0, W=32, H=32, cx=None, cy=None, cam=None):
    """One env with the given nodes (slot j = node j) and one pinhole camera."""
    poses = poses if poses is not None else [IDENT] * len(nodes)
    cam = cam if cam is not None else IDENT
    cx = W / 2.0 if cx is None else cx
    cy = H / 2.0 if cy is None else cy
    sc = S.scene_from_lists("hand", list(nodes), [list(range(len(nodes)))], [list(poses)],
                            [[(f, f, cx, cy, W, H, cam)]])
    # keep the exact (float64) poses: closed-form checks must not see float32 rounding
    sc.node_poses = np.stack([np.asarray(P, np.float64) for P in poses])[None]
    sc.cam_pose = np.asarray(cam, np.float64)[None, None]
    sc.cam_intr = np.array([[[f, f, cx, cy]]], np.float64)
    return sc


def rigid(R, t):
    return np.concatenate([np.asarray(R, np.float64), np.asarray(t, np.float64).reshape(3, 1)], axis=1)


def compose(A, B):
    """[R|t] of A o B for 3x4 rigid transforms."""
    RA, tA, RB, tB = A[:, :3], A[:, 3], B[:, :3], B[:, 3]
    return rigid(RA @ RB, RA @ tB + tA)


def inverse(A):
    R, t = A[:, :3], A[:, 3]
    return rigid(R.T, -R.T @ t)
