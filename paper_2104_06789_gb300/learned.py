"""Learned proposal: training windows, plain-EM labels, training with the
library's BF16 tensor-core kernels, and the comparison of the plain and the
learned initialisation.

Scenes: the handheld family of synthetic.handheld (planar patches and boxes
in [0.5, 8] m, per-frame |t| <= 0.05 m and rotation <= 5 deg, 20 % non-rigid
pixels), rendered at the driving image size 1242x375, f = 718 px, T = 8, so
that the network reads 2T = 16 flow channels. Training windows take scene
seeds 5000 + i, held-out windows 9000 + i; the flows are stored as FP16, as
the EM reads them.

Labels: the plain EM's state after `label_iters` iterations from the
triangulation bootstrap: target log-depth = log(theta) minus its median over
the pixels strictly inside the depth range (the network predicts depth up to
the scale that T_1 fixes at bootstrap), target rigidness = mean over the
frames of W_t.

Comparison: for every held-out window, the pose error after k = 1..K EM
iterations from (a) the triangulation bootstrap and (b) the learned bootstrap.
Pose error = mean over the frames of |t_est - t_true| in metres (the rotation
error in degrees is reported beside it). The learned initialisation's
iterations to the plain EM's error = the smallest k at which its mean error
over the held-out set is within 1 % of the plain EM's after `plain_iters`
iterations; its wall time = bootstrap time + k times the time of one
iteration, both measured with CUDA events on the window's stream.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os
import time

import numpy as np

from . import synthetic, voldor

SCENE = dict(W=1242, H=375, f=718.0, T=8)
TRAIN_SEED0, HELDOUT_SEED0 = 5000, 9000


def scene(seed, W=SCENE["W"], H=SCENE["H"], f=SCENE["f"], T=SCENE["T"]):
    """One window of the training family: (flows FP16 [T][H][W][2], K,
    poses [T][4][4], depth0 [H][W], inverse-depth range)."""
    w = synthetic.handheld(seed=seed, W=W, H=H, f=f, T=T)
    return w.flows.astype(np.float16), w.K, w.poses, w.depth0.astype(np.float32), w.inv_depth_range


def _scene_args(args):
    return scene(*args)


def scenes(seeds, workers=0, **size):
    """Yields scene(seed) for the seeds in order, generated by `workers`
    spawned processes (0: in this process)."""
    jobs = [(s, size.get("W", SCENE["W"]), size.get("H", SCENE["H"]), size.get("f", SCENE["f"]),
             size.get("T", SCENE["T"])) for s in seeds]
    if workers <= 0:
        for j in jobs:
            yield _scene_args(j)
        return
    # one BLAS thread per worker: the workers already fill the cores
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        pool = mp.get_context("spawn").Pool(workers)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    with pool:
        yield from pool.imap(_scene_args, jobs, chunksize=1)


def pose_errors(P, gt):
    """(mean translation error in metres, mean rotation error in degrees)."""
    dt = np.linalg.norm(P[:, :3, 3] - gt[:, :3, 3], axis=1)
    c = (np.einsum("tij,tij->t", P[:, :3, :3], gt[:, :3, :3]) - 1.0) / 2.0
    ang = np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))
    return float(dt.mean()), float(ang.mean())


class Dataset:
    """Flows [N][T][H][W][2] FP16 and targets [N][H][W][2] FP32 on the device,
    plus the scenes' poses and depths on the host."""

    def __init__(self, n, T, H, W, device="cuda"):
        import torch
        self.flows = torch.empty((n, T, H, W, 2), dtype=torch.float16, device=device)
        self.targets = torch.empty((n, H, W, 2), dtype=torch.float32, device=device)
        self.poses = np.zeros((n, T, 4, 4))
        self.depth0 = np.zeros((n, H, W), np.float32)
        self.n = 0

    def add(self, flows16, poses, depth0):
        import torch
        i = self.n
        self.flows[i].copy_(torch.from_numpy(flows16))
        self.poses[i] = poses
        self.depth0[i] = depth0
        self.n += 1
        return i


def make_params(inv_range, S):
    return voldor.default_params(inv_depth_min=inv_range[0], inv_depth_max=inv_range[1], hyps_per_frame=S)


def init_weights(T, seed=0, width=32):
    """He-normal weights (std sqrt(2 / (9 Cin))) and zero biases in the
    parameter layout of voldor_net_set_weights."""
    rng = np.random.default_rng(seed)
    cin = [2 * T] + [width] * 5
    cout = [width] * 5 + [2]
    parts = []
    for ci, co in zip(cin, cout):
        parts.append(rng.normal(0.0, math.sqrt(2.0 / (9 * ci)), size=co * 9 * ci))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def build_dataset(seeds, S=4096, label_iters=8, workers=0, log=None, **size):
    """Generates the windows and, if label_iters > 0, runs the plain EM on each
    and stores its labels."""
    import torch
    win = ds = None
    t0 = time.time()
    for i, (f16, K, poses, depth0, inv_range) in enumerate(scenes(seeds, workers, **size)):
        T, H, W = f16.shape[:3]
        if ds is None:
            ds = Dataset(len(seeds), T, H, W)
        j = ds.add(f16, poses, depth0)
        if label_iters <= 0:
            continue
        if win is None:
            win = voldor.Window(ds.flows[j], K, make_params(inv_range, S))
        else:
            win.set_flows(ds.flows[j])
        win.bootstrap(poses[0])
        win.em_step(label_iters)
        _, D, Wm = win.get_pose_depth_rigidness(poses=False)
        ld = np.log(np.maximum(D, 1e-6))
        inside = (D > 1.0001 / inv_range[1]) & (D < 0.9999 / inv_range[0])
        ld = ld - (np.median(ld[inside]) if inside.any() else np.median(ld))
        tgt = np.stack([ld, Wm.mean(axis=0)], -1).astype(np.float32)
        ds.targets[j].copy_(torch.from_numpy(tgt))
        if log and (i + 1) % 100 == 0:
            log(f"labelled {i + 1}/{len(seeds)} windows in {time.time() - t0:.0f} s")
    if win is not None:
        win.destroy()
    return ds


def train(net, ds, steps, batch=2, lr=1e-3, lr_min=1e-5, lam_r=1.0, seed=0, log=None):
    """Adam with a cosine learning rate on random runs of `batch` consecutive
    training windows (whole images). Returns the loss per step."""
    rng = np.random.default_rng(seed)
    losses = np.zeros(steps)
    for s in range(steps):
        lr_s = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * s / steps))
        i = int(rng.integers(0, ds.n - batch + 1))
        losses[s] = net.train_step(ds.flows[i:i + batch], ds.targets[i:i + batch], lr_s, lam_r)
        if log and (s + 1) % 500 == 0:
            log(f"step {s + 1}/{steps}: loss {losses[max(0, s - 99):s + 1].mean():.4f}")
    return losses


MODES = {"plain": None, "learned": dict(depth=True, rigidness=True), "learned_w": dict(depth=False, rigidness=True)}


def compare(net, ds, S=4096, max_iters=8, plain_iters=5, inv_range=(1 / 16.0, 1 / 0.25), K=None):
    """Pose error and time of the plain initialisation, the learned one, and
    the learned rigidness prior over the triangulated depth ("learned_w") on
    the windows of `ds` (see the module docstring)."""
    import torch
    n = ds.n
    T, H, W = ds.flows.shape[1:4]
    if K is None:
        K = (SCENE["f"], SCENE["f"], (W - 1) / 2.0, (H - 1) / 2.0)
    win = voldor.Window(ds.flows[0], K, make_params(inv_range, S))
    err = {m: np.zeros((n, max_iters + 1, 2)) for m in MODES}
    depth_err = {m: np.zeros(n) for m in MODES}
    t_boot = {m: [] for m in MODES}
    t_iter = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for i in range(n):
        win.set_flows(ds.flows[i])
        gt = ds.poses[i]
        ok = np.isfinite(ds.depth0[i]) & (ds.depth0[i] > 0)
        for mode, how in MODES.items():
            torch.cuda.synchronize()
            ev[0].record()
            if how is None:
                win.bootstrap(gt[0])
            else:
                net.bootstrap(win, gt[0], **how)
            ev[1].record()
            torch.cuda.synchronize()
            t_boot[mode].append(ev[0].elapsed_time(ev[1]))
            P, D, _ = win.get_pose_depth_rigidness(rigidness=False)
            err[mode][i, 0] = pose_errors(P, gt)
            depth_err[mode][i] = float(np.median(np.abs(np.log(D[ok]) - np.log(ds.depth0[i][ok]))))
            for k in range(1, max_iters + 1):
                ev[0].record()
                win.em_step(1)
                ev[1].record()
                torch.cuda.synchronize()
                t_iter.append(ev[0].elapsed_time(ev[1]))
                P, _, _ = win.get_pose_depth_rigidness(depth=False, rigidness=False)
                err[mode][i, k] = pose_errors(P, gt)
    win.destroy()
    mean = {m: err[m].mean(axis=0) for m in err}
    target = mean["plain"][plain_iters, 0]
    it_ms = float(np.median(t_iter))
    boot = {m: float(np.median(t_boot[m])) for m in t_boot}
    out = {"windows": n, "S": S, "plain_iters": plain_iters, "target_err_m": float(target),
           "iteration_ms": it_ms, "bootstrap_ms": boot,
           "init_depth_log_err": {m: float(np.median(depth_err[m])) for m in depth_err},
           "plain_ms": boot["plain"] + plain_iters * it_ms}
    med = {m: np.median(err[m], axis=0) for m in err}
    out["median_target_err_m"] = float(med["plain"][plain_iters, 0])
    for m in MODES:
        out[f"{m}_err_m"] = [float(v) for v in mean[m][:, 0]]
        out[f"{m}_rot_deg"] = [float(v) for v in mean[m][:, 1]]
        out[f"{m}_median_err_m"] = [float(v) for v in med[m][:, 0]]
        out[f"{m}_median_rot_deg"] = [float(v) for v in med[m][:, 1]]
        # windows whose error after plain_iters iterations exceeds 10 cm
        out[f"{m}_failures"] = int(np.sum(err[m][:, plain_iters, 0] > 0.1))
        out[f"{m}_per_window_err_m"] = [[float(v) for v in err[m][i, :, 0]] for i in range(n)]
        if m == "plain":
            continue
        k_m = next((k for k in range(max_iters + 1) if mean[m][k, 0] <= 1.01 * target), None)
        k_med = next((k for k in range(max_iters + 1) if med[m][k, 0] <= 1.01 * med["plain"][plain_iters, 0]), None)
        out[f"{m}_median_iters_to_target"] = k_med
        out[f"{m}_median_ms"] = None if k_med is None else boot[m] + k_med * it_ms
        out[f"{m}_iters_to_target"] = k_m
        out[f"{m}_ms"] = None if k_m is None else boot[m] + k_m * it_ms
        out[f"{m}_per_window_reached"] = float(np.mean([
            any(err[m][i, k, 0] <= 1.01 * err["plain"][i, plain_iters, 0] for k in range(plain_iters + 1))
            for i in range(n)]))
    return out
