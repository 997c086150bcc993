"""Sliding-window visual odometry over a flow sequence.

The paper runs its inference on batches of 4-8 flows and, for a sequence,
initialises T_1 of a batch from the previous estimates when consecutive
batches overlap (Sec. 5.3; KITTI with batches of 6 flows, Sec. 6.1). This
driver does that over the C ABI with one reused window context:

- window k covers the flows X_{s+1} .. X_{s+T} of frames s .. s+T, s = k * stride
  (1 <= stride <= T - 1, so consecutive windows overlap by T - stride flows);
- the first window's T_1 is the caller's, or the epipolar estimate of X_1 with
  |t| = the caller's baseline; window k+1's T_1 is window k's estimate of the
  relative pose of frames s+stride -> s+stride+1 (its T_{stride+1}), which
  carries the scale from window to window;
- window k contributes its first `stride` relative poses to the trajectory (the
  last window contributes all of its remaining ones);
- the trajectory is chained as world-to-camera transforms M_0 = I,
  M_{f+1} = T_{f+1} M_f (T_f maps camera f-1 coordinates to camera f);
- with a camera height, every window's depth and translations are rescaled
  after its EM so that its ground plane lies that far below the camera
  (Sec. 6.1's absolute scale from the ground plane), instead of inheriting the
  scale of the window before.
"""
from __future__ import annotations

import numpy as np

from . import voldor


def window_starts(n_flows, T, stride):
    """First frame of every window; the last window ends at the last flow."""
    if not (1 <= T <= n_flows):
        raise ValueError("window length must be in [1, number of flows]")
    if T > 1 and not (1 <= stride <= T - 1):
        raise ValueError("stride must be in [1, T - 1] so that windows overlap")
    starts = list(range(0, n_flows - T + 1, stride if T > 1 else 1))
    if starts[-1] != n_flows - T:
        starts.append(n_flows - T)
    return starts


def chain(relative):
    """World-to-camera transforms M_0..M_n from relative poses T_1..T_n."""
    M = [np.eye(4)]
    for T in relative:
        M.append(np.asarray(T) @ M[-1])
    return np.array(M)


class SlidingWindowVO:
    """Runs the EM on overlapping windows of a flow sequence.

    `make_window(flows, K, params)` builds the window context (the library's
    `voldor.Window` by default; tests pass a stand-in)."""

    def __init__(self, K, T=6, stride=1, n_iters=5, params=None, make_window=None):
        self.K = tuple(float(v) for v in K)
        self.T = int(T)
        self.stride = int(stride)
        self.n_iters = int(n_iters)
        self.params = params
        self.make_window = make_window or (lambda f, K, p: voldor.Window(f, K, p))

    def run(self, flows, T1=None, baseline=1.0, epi_samples=512, camera_height=None, max_tilt_deg=10.0):
        """flows [n][H][W][2] (numpy or torch, FP16 or FP32). Returns a dict:
        `relative` [n][4][4] (T_1..T_n), `trajectory` [n+1][4][4]
        (world-to-camera), `starts` (first frame of each window) and
        `window_poses` (each window's estimates)."""
        n = flows.shape[0]
        starts = window_starts(n, self.T, self.stride)
        win = None
        relative = [None] * n
        window_poses = []
        next_T1 = None if T1 is None else np.asarray(T1, dtype=np.float64)
        for k, s in enumerate(starts):
            sub = flows[s:s + self.T]
            if win is None:
                win = self.make_window(sub, self.K, self.params)
            else:
                win.set_flows(sub)
            if next_T1 is None:
                next_T1 = win.bootstrap_epipolar(epi_samples, baseline)
            else:
                win.bootstrap(next_T1)
            win.em_step(self.n_iters)
            if camera_height is not None:
                win.ground_scale(camera_height, max_tilt_deg, apply=True)
            P, _, _ = win.get_pose_depth_rigidness(depth=False, rigidness=False)
            window_poses.append(P)
            last = k == len(starts) - 1
            keep_to = self.T if last else (starts[k + 1] - s)
            for i in range(keep_to):
                if relative[s + i] is None:
                    relative[s + i] = P[i]
            if not last:
                step = starts[k + 1] - s
                next_T1 = P[step] if step < self.T else P[-1]
        if hasattr(win, "destroy"):
            win.destroy()
        rel = np.array(relative)
        return dict(relative=rel, trajectory=chain(rel), starts=starts, window_poses=window_poses)
