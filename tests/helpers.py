"""Shared test fixtures: seeded windows and state transfer between the CUDA
library and the oracle (inputs only; no expected values come from the CUDA
path)."""
import numpy as np

from paper_2104_06789_gb300 import synthetic as sy


def small_window(seed=1000, **kw):
    return sy.small_planes(seed=seed, **kw)


def rotation_angle(Ra, Rb):
    c = (np.trace(Ra @ Rb.T) - 1.0) / 2.0
    return float(np.arccos(np.clip(c, -1.0, 1.0)))


def pose_close(Pa, Pb, rad=1e-6, rel=1e-6):
    ang = rotation_angle(Pa[:3, :3], Pb[:3, :3])
    dt = np.linalg.norm(Pa[:3, 3] - Pb[:3, 3]) / max(np.linalg.norm(Pb[:3, 3]), 1e-12)
    return ang <= rad and dt <= rel, ang, dt


def f32_state(rng, w, depth=None):
    """A teacher-forcing state whose values are exactly representable in FP32."""
    if depth is None:
        depth = w.depth0 * rng.uniform(0.9, 1.1, size=w.depth0.shape)
    depth = depth.astype(np.float32)
    rig = rng.uniform(0.0, 1.0, size=(w.T, w.H, w.W)).astype(np.float32)
    return depth, rig


def oracle_window(oracle, w, flows64, S, depth32, rig32, poses, **kw):
    ow = oracle.OracleWindow(flows64, w.K, S=S, inv_depth_min=w.inv_depth_range[0],
                             inv_depth_max=w.inv_depth_range[1], **kw)
    ow.theta[:] = depth32.astype(np.float64)
    ow.wmap[:] = rig32.astype(np.float64)
    ow.poses[:] = poses
    return ow


def f32_hypotheses(rng, R0, t0, n, rot=0.02, trans=0.02):
    """Hypotheses near (R0, t0) whose scoring form R - I, t is exact in FP32."""
    Rs, ts = [], []
    for i in range(n):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        a = rng.uniform(0, rot) if i else 0.0
        Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        R = (np.eye(3) + np.sin(a) * Kx + (1 - np.cos(a)) * Kx @ Kx) @ R0
        t = t0 + (rng.normal(size=3) * trans if i else 0.0)
        E = (R - np.eye(3)).astype(np.float32).astype(np.float64)
        Rs.append(np.eye(3) + E)
        ts.append(t.astype(np.float32).astype(np.float64))
    return np.array(Rs), np.array(ts)


def tie_runs(ow, k, q, th0, lab_ref, lab_gpu, margin=1e-5):
    """Pixels whose sweep decision FP32 scoring cannot be held to: walking each
    chain in the sweep's order, a pixel where the oracle's best two candidate
    scores (prev, the carried neighbour, the depth sample) are within `margin`
    relative (the per-pixel likelihood tolerance) starts a tie, and the pixels
    after it stay tied while either side carries its neighbour's value (label
    1); the first pixel where both sides take their own value ends it. Every
    other pixel's label and depth must equal the oracle's."""
    H, W = th0.shape
    rows = k % 2 == 0
    n_ch, ln = (H, W) if rows else (W, H)
    tied = np.zeros((H, W), bool)
    for c in range(n_ch):
        carried, run = None, False
        for i in range(ln):
            x, y = [(i, c), (c, i), (W - 1 - i, c), (c, H - 1 - i)][k % 4]
            j = y * W + x
            sc = [ow.mie_score(q, j, float(th0[y, x])), ow.mie_score(q, j, ow.depth_sample(k, j))]
            if carried is not None:
                sc.append(ow.mie_score(q, j, carried))
            sc = sorted(sc, reverse=True)
            tie = len(sc) > 1 and sc[0] - sc[1] <= margin * abs(sc[0])
            if tie:
                run = True
            elif lab_ref[y, x] != 1 and lab_gpu[y, x] != 1:
                run = False
            tied[y, x] = run
            carried = float(ow.theta[y, x])
    return tied
