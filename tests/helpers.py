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
