"""Hypothesis-count autotuning of a window.

The dense scoring's cost is linear in S, the number of P3P hypotheses kept per
frame, while the pose the meanshift returns stops improving once S is large
enough for the window's geometry. Because the groups are drawn from the
window's Philox stream in a fixed order and collected until S solutions are
found, the hypotheses of a smaller S are a prefix of those of a larger one.

`autotune_hyps` runs the window from the same bootstrap, `iters` EM iterations
each, with the largest hypothesis count (`params.hyps_per_frame`) and with
each smaller candidate, and returns the smallest candidate whose poses agree
with the largest's on every frame. By default the agreement bound is the
estimator's own Monte-Carlo spread: the largest count is run a second time
with another Philox key, and a candidate is accepted when it is no farther
from the reference run (rotation angle, translation difference relative to
the reference translation) than that second full run is. Explicit bounds
(`rot_tol` radians, `trans_tol` relative) replace the measured spread. The
tile shape of the dense scoring is tuned afterwards on the chosen count
(`Window.autotune`).
"""
from __future__ import annotations

import numpy as np

from . import voldor


def pose_agreement(P, Q):
    """(max rotation angle in radians, max translation difference relative to
    the norm of Q's translation) over the frames of two [T][4][4] stacks."""
    c = (np.einsum("tij,tij->t", P[:, :3, :3], Q[:, :3, :3]) - 1.0) / 2.0
    ang = np.arccos(np.clip(c, -1.0, 1.0))
    dt = np.linalg.norm(P[:, :3, 3] - Q[:, :3, 3], axis=1)
    ref = np.maximum(np.linalg.norm(Q[:, :3, 3], axis=1), 1e-12)
    return float(ang.max()), float((dt / ref).max())


def default_candidates(S):
    """S/8, S/4, S/2 (at least 64), ascending."""
    return sorted({max(64, S // d) for d in (8, 4, 2)} - {S})


def autotune_hyps(flows, K, params, T1, candidates=None, iters=5, rot_tol=None, trans_tol=None,
                  make_window=None):
    """Returns (chosen hypothesis count, [(S, rotation disagreement,
    relative translation disagreement) per candidate tried], (rotation bound,
    translation bound)). `make_window(flows, K, params)` builds a window (the
    library's `voldor.Window` by default)."""
    make_window = make_window or (lambda f, k, p: voldor.Window(f, k, p))
    S_max = int(params.hyps_per_frame)
    cands = sorted(int(s) for s in (candidates if candidates is not None else default_candidates(S_max)))
    if any(s < 1 or s > S_max for s in cands):
        raise ValueError("candidate hypothesis counts must be in [1, params.hyps_per_frame]")

    def run(S, seed_offset=0):
        p = type(params).from_buffer_copy(params)
        p.hyps_per_frame = S
        p.groups_per_frame = max(int(params.groups_per_frame) * S // S_max, 1)
        p.seed = (int(params.seed) + seed_offset) % (1 << 64)
        w = make_window(flows, K, p)
        try:
            w.bootstrap(T1)
            w.em_step(iters)
            P, _, _ = w.get_pose_depth_rigidness(depth=False, rigidness=False)
        finally:
            if hasattr(w, "destroy"):
                w.destroy()
        return P

    ref = run(S_max)
    if rot_tol is None or trans_tol is None:
        spread_rot, spread_trans = pose_agreement(run(S_max, seed_offset=1), ref)
        rot_tol = spread_rot if rot_tol is None else rot_tol
        trans_tol = spread_trans if trans_tol is None else trans_tol
    tried = []
    for S in cands:
        if S == S_max:
            break
        ang, rel = pose_agreement(run(S), ref)
        tried.append((S, ang, rel))
        if ang <= rot_tol and rel <= trans_tol:
            return S, tried, (rot_tol, trans_tol)
    return S_max, tried, (rot_tol, trans_tol)
