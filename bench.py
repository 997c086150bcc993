#!/usr/bin/env python
"""Throughput of VOLDOR's generalized-EM loop on one GB300 per rank.

A step is one whole window: bootstrap (triangulation from the given T_1) and
5 EM iterations (for each of the T frames: minimal groups, P3P, dense scoring
of every hypothesis against every pixel, meanshift; then E-step smoothing,
MIE depth sweep, rigidness update) on the seeded 1242x375, T=8 driving-like
window with FP16 flows and 8192 pose hypotheses per frame.

  value   Mpixel*frame EM updates per second = H*W*T*iters / step time, with the
          flows already resident in HBM; whole job (sum over ranks of units
          / max over ranks of time).
  e2e     the same through the C ABI with host buffers: host->device copy of
          the flows (pinned), bootstrap, EM, device->host read of poses, depth
          and rigidness, all inside the timed step.

Multi-GPU: windows are independent, so ranks run replicas on their own
windows (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel·frame EM updates/s at 1242x375 T=8; learned vs plain time-to-equal-pose-error"
UNIT = "Mpixel*frame/s"
MUFU_PER_SM_PER_CLK = 16          # 4 SFU lanes per SM sub-partition, 4 sub-partitions
# algorithmic SFU operations per hypothesis-pixel pair, (rcp, lg2, ex2), by
# (criterion, residual model): the projection's reciprocal; Fisk: lg2 + ex2 for
# (x/alpha)^beta and lg2 of 1 + mu/rho (MIE) or of mu/rho (MLE); Gaussian:
# log2(mu/rho) is linear in x, MIE adds ex2 + lg2 for log2(1 + 2^-|s|)
ALGO_MUFU_MIX = {("mie", "fisk"): (1, 2, 1), ("mle", "fisk"): (1, 2, 1),
                 ("mie", "gaussian"): (1, 1, 1), ("mle", "gaussian"): (1, 0, 0)}
NOMINAL_SMS, NOMINAL_MAX_MHZ = 152, 2070.0
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per k_score launch,
# mean over the 40 launches of one driving-window step (S = 8192 on every frame,
# 5 iterations), from one ncu capture of the current default MIE / Fisk kernel
# (2 hypotheses per thread, three blocks per SM), over two complete iterations:
# 14.19 MB read, < 1 KB written, against 48 B per valid record + 48 B per
# hypothesis of algorithmic bytes (13.8 MB at the mean of ~280k valid pixels
# per frame; frame 1: 23.32 MB read for 22.75 MB). The other
# variants and hypothesis counts were not captured: their traffic is null.
SCORE_TRAFFIC_BYTES = {("mie", "fisk", 8192): 14.19e6}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--iters", type=int, default=5)
    ap.add_argument("--hyps", type=int, default=8192)
    ap.add_argument("--criterion", choices=["mie", "mle"], default="mie",
                    help="depth and pose criterion (MLE: the ablation variant)")
    ap.add_argument("--residual", choices=["fisk", "gaussian"], default="fisk",
                    help="flow residual model (Gaussian: the ablation variant)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched (config 4) and learned-vs-plain (config 5) measurements of the default line")
    ap.add_argument("--batch", type=int, default=0,
                    help="run the batched workload instead: this many windows of mixed size and T in one graph")
    ap.add_argument("--learned", type=int, default=0,
                    help="run the learned-proposal comparison instead: train on this many windows")
    ap.add_argument("--heldout", type=int, default=64)
    ap.add_argument("--train-steps", type=int, default=20000)
    ap.add_argument("--workers", type=int, default=0, help="scene-generator processes (0: cpu count - 1)")
    ap.add_argument("--save-weights", default="")
    ap.add_argument("--weights", default="", help="with --learned: evaluate these weights instead of training")
    ap.add_argument("--probe-sfu", action="store_true",
                    help="print the SFU probe's results per SM clock (exp2, log2, rcp) and exit")
    ap.add_argument("--net", type=int, default=0,
                    help="time the proposal network instead: forward passes on this many 1242x375 T=8 flow stacks")
    return ap.parse_args()


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def workload(rank):
    from paper_2104_06789_gb300 import synthetic
    return synthetic.driving(seed=3000 + rank)


def max_over_ranks(x, dist, device):
    """The maximum of a per-rank float over all ranks (x itself on one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, max_seconds):
    """Units of all ranks over the slowest rank's time, in millions per second
    (replicas: every rank processes the same number of units)."""
    return world * units_per_rank / max_seconds / 1e6


def config_dict(w, args, world):
    return {"workload": w.name, "width": w.W, "height": w.H, "T": w.T, "em_iters": args.iters,
            "hyps_per_frame": args.hyps, "groups_per_frame": 4 * args.hyps, "flows": "fp16",
            "focal_px": w.K[0], "windows_per_rank": 1, "parallelism": f"replicas x{world}",
            "l2": "flushed between timed steps (256 MiB write)",
            "criterion": args.criterion, "residual": args.residual}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = np.array([r[0] for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(r[1] for r in rows)),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the same window
# ---------------------------------------------------------------------------
def variant_overrides(args):
    """Oracle parameters of the variant `args` selects (criterion 1 = MLE,
    residual 1 = Gaussian; 0 the paper's MIE and Fisk model)."""
    return {"criterion": int(args.criterion == "mle"), "residual": int(args.residual == "gaussian")}


def _scored(hyps_scored, T, S):
    """Hypotheses scored on frames 1..T (the GPU's per-frame counts, S when
    not given)."""
    return [S] * T if hyps_scored is None else [float(h) for h in hyps_scored]


def oracle_sample(w, S, iters, n_score_hyps=4, variant=None, hyps_scored=None):
    """Times the FP64 oracle on one EM iteration of window `w`: dense scoring
    of n_score_hyps hypotheses per frame, scaled linearly (its cost is linear
    in the count) to the hypotheses the GPU scored on that frame; the minimal
    groups, P3P and collection of S hypotheses per frame, timed whole; one
    pass of the per-pixel steps (E-step, MIE sweep, rigidness), timed whole.
    Returns (Mpixel*frame/s, seconds of CPU work, description)."""
    import oracle
    oracle.build()
    flows = w.flows.astype(np.float16).astype(np.float64)
    ow = oracle.OracleWindow(flows, w.K, S=S, G=4 * S, inv_depth_min=w.inv_depth_range[0],
                             inv_depth_max=w.inv_depth_range[1], **(variant or {}))
    ow.bootstrap(w.poses[0])
    scored = _scored(hyps_scored, w.T, S)
    t_score = []
    for t in range(1, w.T + 1):
        R = np.tile(w.poses[t - 1][:3, :3], (n_score_hyps, 1, 1))
        tv = np.tile(w.poses[t - 1][:3, 3], (n_score_hyps, 1))
        t0 = time.perf_counter()
        ow.score(t, R, tv)
        t_score.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    n_col = [len(ow.collect_hypotheses(0, t)[0]) for t in range(1, w.T + 1)]
    t_groups = time.perf_counter() - t0
    t0 = time.perf_counter()
    em = ow.emissions()
    q = ow.smooth(0, em)
    ow.mie_sweep(0, q)
    ow.rigidness()
    t_pixel = time.perf_counter() - t0
    score_full = sum(ts * n / n_score_hyps for ts, n in zip(t_score, scored))
    per_iter = score_full + t_groups + t_pixel
    measured = sum(t_score) + t_groups + t_pixel
    value = w.H * w.W * w.T / per_iter / 1e6
    desc = (f"one EM iteration of the same window: dense scoring timed on {n_score_hyps} hypotheses x {w.T} "
            f"frames and scaled to the {sum(scored) / w.T:.0f} hypotheses per frame the GPU scored; minimal groups, "
            f"P3P and collection timed whole ({min(n_col)}-{max(n_col)} hypotheses per frame); E-step + MIE sweep + "
            f"rigidness timed whole; {per_iter:.1f} s/iteration extrapolated from {measured:.1f} s measured")
    return value, measured, desc


def _oracle_piece(args):
    """One process's share of the parallel oracle sample: dense scoring of the
    sampled hypotheses and the collection of frame t's S hypotheses.
    Returns (scoring seconds, collection seconds)."""
    flows16, K, poses, inv_range, t, n_score_hyps, S, variant = args
    import oracle
    flows = flows16.astype(np.float64)
    ow = oracle.OracleWindow(flows, K, S=S, G=4 * S, inv_depth_min=inv_range[0], inv_depth_max=inv_range[1],
                             **variant)
    ow.bootstrap(poses[0])
    R = np.tile(poses[t - 1][:3, :3], (n_score_hyps, 1, 1))
    tv = np.tile(poses[t - 1][:3, 3], (n_score_hyps, 1))
    t0 = time.perf_counter()
    ow.score(t, R, tv)
    t_score = time.perf_counter() - t0
    t0 = time.perf_counter()
    ow.collect_hypotheses(0, t)
    return t_score, time.perf_counter() - t0


def oracle_sample_parallel(w, S, iters, workers, n_score_hyps=4, variant=None, hyps_scored=None):
    """The same sample as oracle_sample with its independent pieces (each
    frame's dense scoring and collection) on `workers` spawned processes,
    each running the unchanged single-threaded oracle; the per-pixel passes
    (one sequential pass each) stay on one core. Returns (Mpixel*frame/s,
    wall seconds, description, processes)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    f16 = w.flows.astype(np.float16)
    jobs = [(f16, w.K, w.poses, w.inv_depth_range, t, n_score_hyps, S, variant or {})
            for t in range(1, w.T + 1)]
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(min(workers, len(jobs))) as pool:
            pool.map(_oracle_piece, jobs[:1])                      # start-up outside the timed region
            t0 = time.perf_counter()
            parts = pool.map(_oracle_piece, jobs)
            t_par = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    scored = _scored(hyps_scored, w.T, S)
    t_score = sum(p[0] * n / n_score_hyps for p, n in zip(parts, scored))
    t_groups = sum(p[1] for p in parts)
    n_proc = min(workers, len(jobs))
    flows = f16.astype(np.float64)
    ow = oracle.OracleWindow(flows, w.K, S=S, G=4 * S, inv_depth_min=w.inv_depth_range[0],
                             inv_depth_max=w.inv_depth_range[1], **(variant or {}))
    ow.bootstrap(w.poses[0])
    t0 = time.perf_counter()
    em = ow.emissions()
    q = ow.smooth(0, em)
    ow.mie_sweep(0, q)
    ow.rigidness()
    t_pixel = time.perf_counter() - t0
    # the frames' pieces are independent, and a frame's dense scoring splits
    # into hypothesis blocks: spread evenly over the processes
    per_iter = (t_score + t_groups) / n_proc + t_pixel
    value = w.H * w.W * w.T / per_iter / 1e6
    desc = (f"one EM iteration of the same window on {n_proc} processes (spawned, one thread each, the unchanged "
            f"oracle): dense scoring ({n_score_hyps} hypotheses x {w.T} frames measured, scaled to the "
            f"{sum(scored) / w.T:.0f} per frame the GPU scored) and the collection of S hypotheses per frame "
            f"(timed whole) split evenly over the processes, E-step + MIE sweep + rigidness on one core; "
            f"{per_iter:.1f} s/iteration extrapolated from {t_par + t_pixel:.1f} s measured")
    return value, t_par + t_pixel, desc, n_proc


def _f32_hypotheses(rng, R0, t0, n, rot=0.02, trans=0.02):
    """n hypotheses near (R0, t0) whose scoring form (R - I, t) is exact in
    FP32, so that both sides score the same poses."""
    Rs, ts = [], []
    for i in range(n):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        a = rng.uniform(0, rot) if i else 0.0
        Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        R = (np.eye(3) + np.sin(a) * Kx + (1 - np.cos(a)) * Kx @ Kx) @ R0
        E = (R - np.eye(3)).astype(np.float32).astype(np.float64)
        Rs.append(np.eye(3) + E)
        ts.append((t0 + (rng.normal(size=3) * trans if i else 0.0)).astype(np.float32).astype(np.float64))
    return np.array(Rs), np.array(ts)


def error_vs_oracle(win, w, flows16, params, variant, n_hyps=8, k=1):
    """Per-result error of the GPU against the FP64 oracle on the window's
    final state (depth, rigidness and poses after the timed steps, read back
    and handed to the oracle exactly): dense scores L_h of n_hyps hypotheses
    of the last frame (relative); every per-pixel log-likelihood ell = log W
    of the rigidness update (relative, with the FP32 storage of W); the depth
    sweep's labels (agreement); the last frame's pose update (identical
    hypothesis set, then the oracle's meanshift on the GPU's hypotheses and
    seed: rotation angle and relative translation of the result)."""
    import oracle
    oracle.build()
    P, D, Wm = win.get_pose_depth_rigidness()
    ow = oracle.OracleWindow(flows16.astype(np.float64), w.K, S=params.hyps_per_frame, G=params.groups_per_frame,
                             inv_depth_min=params.inv_depth_min, inv_depth_max=params.inv_depth_max,
                             seed=params.seed, window_id=params.window_id, **variant)
    ow.theta[:] = D.astype(np.float64)
    ow.wmap[:] = Wm.astype(np.float64)
    ow.poses[:] = P
    out = {}
    t = w.T
    rng = np.random.default_rng(5)
    R, tv = _f32_hypotheses(rng, P[t - 1][:3, :3], P[t - 1][:3, 3], n_hyps)
    Lg, Lo = win.score_hypotheses(t, R, tv), ow.score(t, R, tv)
    out["score_rel_max"] = float(np.max(np.abs(Lg - Lo) / np.abs(Lo)))
    out["score_hyps"] = n_hyps
    # rigidness update: log W per (t, j)
    win.rigidness_update()
    _, _, W_gpu = win.get_pose_depth_rigidness(poses=False, depth=False)
    ell_ref = np.log(ow.emissions())
    ell_gpu = np.log(W_gpu.astype(np.float64))
    rel = np.abs(ell_gpu - ell_ref) / np.maximum(np.abs(ell_ref), 1e-300)
    out["ell_rel_max"] = float(rel.max())
    out["ell_within_bound"] = float(np.mean(np.abs(ell_gpu - ell_ref) <= 1e-5 * np.abs(ell_ref) + 2.0 ** -23))
    ow.wmap[:] = W_gpu.astype(np.float64)
    # pose update of the last frame
    win.pose_update(k, t)
    hg = win.hypotheses()
    Ro, to, wo, go, so = ow.collect_hypotheses(k, t)
    same = len(go) == len(hg["group"]) and np.array_equal(go, hg["group"]) and np.array_equal(so, hg["slot"])
    out["hyps_identical"] = bool(same and np.array_equal(wo, hg["weight"]))
    out["hyps_collected"] = int(len(hg["group"]))
    p6 = np.array([oracle.se3_log(Rh, th) for Rh, th in zip(hg["R"], hg["t"])])
    it, x = oracle.meanshift(p6, hg["weight"], hg["seed"], params.sigma_t, params.sigma_r, params.ms_max_iter,
                             params.ms_tol)
    Rm, tm = oracle.se3_exp(x)
    Pg, _, _ = win.get_pose_depth_rigidness(depth=False, rigidness=False)
    c = (np.trace(Pg[t - 1][:3, :3] @ Rm.T) - 1.0) / 2.0
    out["pose_rot_rad"] = float(np.arccos(np.clip(c, -1.0, 1.0)))
    out["pose_trans_rel"] = float(np.linalg.norm(Pg[t - 1][:3, 3] - tm) / np.linalg.norm(tm))
    ow.poses[t - 1] = Pg[t - 1]
    # depth sweep on a seeded smoothed rigidness
    q = rng.uniform(0, 1, size=(w.T, w.H, w.W)).astype(np.float32)
    win.set_buffer(voldor_mod().BUF_SMOOTHED, q)
    win.depth_update(k)
    lab_gpu = win.get_buffer(voldor_mod().BUF_LABELS, (w.H, w.W), np.uint8)
    lab_ref = ow.mie_sweep(k, q.astype(np.float64))
    out["sweep_labels_identical"] = float(np.mean(lab_gpu == lab_ref))
    out["tolerances"] = {"score_rel": 1e-5, "ell": "1e-5 |ell| + 2^-23", "labels": 0.999,
                         "pose_rot_rad": 1e-6, "pose_trans_rel": 1e-6}
    return out


def voldor_mod():
    from paper_2104_06789_gb300 import voldor
    return voldor


# ---------------------------------------------------------------------------
# reference arm: the oracle
# ---------------------------------------------------------------------------
def run_reference(args):
    """The oracle on the machine's host cores (its independent pieces over all of
    them, as in oracle_sample_parallel), each step a bounded sample of one EM
    iteration of the same window, scaled to the full configuration."""
    rank, _, world = rank_info()
    if rank != 0:
        return
    w = workload(0)
    steps = []
    desc, n_proc = "", 1
    for i in range(args.warmup + args.steps):
        v, secs, desc, n_proc = oracle_sample_parallel(w, args.hyps, args.iters, os.cpu_count() or 1,
                                                       n_score_hyps=2, variant=variant_overrides(args))
        if i >= args.warmup:
            steps.append(v)
    value = float(np.mean(steps))
    units = w.H * w.W * w.T * args.iters
    ms = units / (value * 1e6) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w, args, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_proc, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def _guarded(fn, *a):
    """fn(*a), or {"error": ...} if it raises (printed to stderr)."""
    try:
        return fn(*a)
    except Exception as e:                    # noqa: BLE001 -- reported, not swallowed
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": f"{type(e).__name__}: {e}"}


def run_ours(args):
    import torch

    from paper_2104_06789_gb300 import build, voldor

    rank, local_rank, world = rank_info()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    w = workload(rank)
    flows16 = np.ascontiguousarray(w.flows.astype(np.float16))
    stream = torch.cuda.Stream()
    params = voldor.default_params(hyps_per_frame=args.hyps,
                                   inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1],
                                   seed=0, window_id=rank,
                                   criterion={"mie": voldor.CRITERION_MIE, "mle": voldor.CRITERION_MLE}[args.criterion],
                                   residual={"fisk": voldor.RESIDUAL_FISK,
                                             "gaussian": voldor.RESIDUAL_GAUSSIAN}[args.residual])
    dev_flows = torch.from_numpy(flows16).to(f"cuda:{local_rank}")
    torch.cuda.synchronize()
    win = voldor.Window(dev_flows, w.K, params, stream=stream)
    T1 = w.poses[0]
    win.enable_timing(True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local_rank}")

    def step():
        win.bootstrap(T1)
        win.em_step(args.iters)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    score_ms, score_pairs, score_hyps = [], [], []
    launches0 = win.kernel_launches()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)          # L2 flush between timed steps (not timed)
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
            ms, pairs, nh = win.get_score_times(with_hyps=True)
            score_ms.extend(ms.tolist())
            score_pairs.extend(pairs.tolist())
            score_hyps.extend(nh.tolist())
        torch.cuda.synchronize()
    launches = win.kernel_launches() - launches0
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist, f"cuda:{local_rank}")
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    units_per_step = w.H * w.W * w.T * args.iters
    value = whole_job_rate(world, units_per_step * args.steps, total_ms / 1e3)

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pinned = torch.from_numpy(flows16).pin_memory()
        host_win = voldor.Window(pinned, w.K, params, stream=stream)
        P = np.zeros((w.T, 4, 4))
        for i in range(args.warmup + args.steps):
            if i == args.warmup:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            host_win.set_flows(pinned)
            host_win.bootstrap(T1)
            host_win.em_step(args.iters)
            P, D, Wm = host_win.get_pose_depth_rigidness()
        e2e_s_max = max_over_ranks(time.perf_counter() - t0, dist, f"cuda:{local_rank}")
        host_win.destroy()
        e2e = {"value": whole_job_rate(world, units_per_step * args.steps, e2e_s_max), "unit": UNIT,
               "h2d_bytes_per_step": int(flows16.nbytes),
               "d2h_bytes_per_step": int(w.T * 16 * 8 + w.H * w.W * 4 + w.T * w.H * w.W * 4)}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    clocks = clk.summary()
    props = torch.cuda.get_device_properties(local_rank)
    sms = props.multi_processor_count
    # the SM clock of the timed region (median of the samples; the maximum
    # clock if none were taken) converts per-clock peaks to rates
    f_mhz = clocks["sm_mhz"] if clocks and clocks.get("sm_mhz") else NOMINAL_MAX_MHZ
    # SFU results per SM clock, measured on this GPU (exp2, log2, reciprocal;
    # whole-grid CUDA-event time over the SM clock measured in the probe),
    # combined over the variant's algorithmic mix per pair
    probe = {name: voldor.probe_sfu_rate(op, with_clock=True) for op, name in enumerate(("ex2", "lg2", "rcp"))}
    rates = {name: r for name, (r, _) in probe.items()}
    mix = dict(zip(("rcp", "lg2", "ex2"), ALGO_MUFU_MIX[(args.criterion, args.residual)]))
    ops_per_pair = sum(mix.values())
    per_clk = ops_per_pair / sum(n / rates[op] for op, n in mix.items())
    peak = sms * per_clk * f_mhz * 1e6 / 1e12                          # T SFU-ops/s
    score_ms = np.array(score_ms)
    score_pairs = np.array(score_pairs, dtype=np.float64)
    # algorithmic work per launch over the mean launch duration (= all timed
    # launches' work over their summed time)
    pair_rate = float(score_pairs.sum() / (score_ms.sum() * 1e-3)) if len(score_ms) else None
    achieved = ops_per_pair * pair_rate / 1e12 if pair_rate else None
    mix_txt = " + ".join(f"{n} {op}" for op, n in mix.items() if n)
    # the log-domain count of the pair term (rcp; lg2 of x; ex2 and lg2 of
    # the softplus in log rho; two for logaddexp): 6 MUFU per pair against
    # the nominal 16 SFU results per SM clock
    nominal_peak = sms * MUFU_PER_SM_PER_CLK * f_mhz * 1e6 / 1e12
    six_op = ({"ops_per_pair": 6, "achieved": 6 * pair_rate / 1e12, "peak": nominal_peak,
               "frac": 6 * pair_rate / 1e12 / nominal_peak,
               "peak_source": f"{sms} SMs x {MUFU_PER_SM_PER_CLK} SFU results/clk/SM (nominal) x {f_mhz:.0f} MHz"}
              if pair_rate and (args.criterion, args.residual) == ("mie", "fisk") else None)
    roofline = {"kernel": "k_score (dense hypothesis scoring)", "bound": "alu", "achieved": achieved,
                "peak": peak, "unit": f"T SFU-op/s ({ops_per_pair} algorithmic SFU ops per hypothesis-pixel pair)",
                "frac": achieved / peak if achieved else None,
                "traffic": SCORE_TRAFFIC_BYTES.get((args.criterion, args.residual, args.hyps)),
                "traffic_unit": "DRAM bytes per launch (ncu)",
                "peak_source": (f"{sms} SMs x {per_clk:.2f} SFU results/clk/SM (measured: ex2 {rates['ex2']:.2f}, "
                                f"lg2 {rates['lg2']:.2f}, rcp {rates['rcp']:.2f} at a probe clock of "
                                f"{probe['rcp'][1]:.0f} MHz; mix {mix_txt}) x {f_mhz:.0f} MHz (timed region)"),
                "six_mufu_per_pair": six_op,
                "launches_timed": int(len(score_ms)), "mean_launch_ms": float(score_ms.mean()) if len(score_ms) else None,
                "share_of_step": float(score_ms.sum() / total_ms) if len(score_ms) else None}
    # hypotheses scored per frame (launch i scores frame i mod T + 1)
    hyps_scored = None
    if score_hyps:
        h = np.array(score_hyps, dtype=np.float64)
        hyps_scored = [float(h[f::w.T].mean()) for f in range(w.T)]

    cpu = cpu_par = None
    if world == 1 and not args.no_cpu:
        v, secs, desc = oracle_sample(w, args.hyps, args.iters, variant=variant_overrides(args),
                                      hyps_scored=hyps_scored)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
        vp, secs_p, desc_p, n_proc = oracle_sample_parallel(w, args.hyps, args.iters, os.cpu_count() or 1,
                                                            variant=variant_overrides(args), hyps_scored=hyps_scored)
        cpu_par = {"value": vp, "unit": UNIT, "cores": n_proc, "kind": "oracle", "sample": desc_p}
    err = None
    if world == 1 and not args.no_cpu:
        err = error_vs_oracle(win, w, flows16, params, variant_overrides(args))
    batch = learned_cmp = None
    if world == 1 and not args.no_extra and (args.criterion, args.residual) == ("mie", "fisk"):
        # measured after the timed region: a failure here is reported in its
        # own object and does not take the headline measurement with it
        batch = _guarded(batch_summary, args.iters, pair_rate)
        learned_cmp = _guarded(learned_summary, args.iters)

    cfg = config_dict(w, args, world)
    if hyps_scored is not None:
        cfg["hyps_scored_per_frame"] = hyps_scored
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg, "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_parallel": cpu_par,
            "e2e": e2e, "error_vs_oracle": err, "gpu_launches": int(launches), "clocks": clocks,
            "batch": batch, "learned_vs_plain": learned_cmp}
    print(json.dumps(line), flush=True)
    win.destroy()
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# batched workload: many windows of mixed resolution and T in one CUDA graph
# ---------------------------------------------------------------------------
def _render_window(job):
    """One window of the mixed batch (module level: runs in spawned workers)."""
    from paper_2104_06789_gb300 import synthetic
    W, H, T, sd = job
    if W == 320:
        return synthetic.small_planes(seed=sd, W=W, H=H, f=0.75 * W, T=T)
    return synthetic.handheld(seed=sd, W=W, H=H, f=0.82 * W, T=T)


def batch_workload(n, seed=4000):
    """n independently rendered windows: resolution uniform over {320x240,
    640x480, 1242x375}, T uniform in [3, 8] and a scene seed of its own each
    (planar-patch scenes at 320x240, handheld scenes otherwise, focal scaled
    with the width). Rendered on spawned processes, one thread each.
    Returns [(window, T)]."""
    import multiprocessing as mp
    rng = np.random.default_rng(seed)
    sizes = [(320, 240), (640, 480), (1242, 375)]
    jobs = []
    for i in range(n):
        W, H = sizes[int(rng.integers(0, 3))]
        jobs.append((W, H, int(rng.integers(3, 9)), seed + 1 + i))
    workers = max(1, min(len(jobs), (os.cpu_count() or 2) - 1))
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            wins = pool.map(_render_window, jobs, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return [(b, job[2]) for b, job in zip(wins, jobs)]


def run_batch(args):
    """Config 4: the batch of mixed windows in one CUDA graph, with the
    hypothesis count of each window autotuned (the smallest of S/8, S/4, S/2
    whose poses after the EM iterations are no farther from S = 4096's than a
    second S = 4096 run with another Philox key is) and then the
    dense-scoring tile shape; the same windows at the fixed S = 4096 are timed
    beside it. Both report the median over windows of the mean translation
    error against the scenes' ground truth. Tuning is not timed."""
    import torch

    from paper_2104_06789_gb300 import build, tuning
    torch.cuda.set_device(0)
    build.build()
    wl = batch_workload(args.batch)
    S = 4096
    fixed, fixed_shapes, _ = _batch_windows(wl, S, args.iters, tune_hyps=False)
    res_f = _batch_measure(fixed, args.iters, None, args.warmup, args.steps)
    tuned, shapes, hyps = _batch_windows(wl, S, args.iters, tune_hyps=True)
    res = _batch_measure(tuned, args.iters, None, args.warmup, args.steps)
    n = len(wl)
    line = {"metric": "windows/s, mixed 320x240/640x480/1242x375 windows, T in [3,8], one CUDA graph",
            "value": res["windows_per_s"], "unit": "windows/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_batch"], "higher_is_better": True,
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": "batch_mixed", "windows": n, "em_iters": args.iters,
                       "hyps_per_frame": f"autotuned per window from {sorted(tuning.default_candidates(S) + [S])}",
                       "flows": "fp16", "resolutions": sorted({f"{b.W}x{b.H}" for b, _ in wl})},
            "autotuned_hyps": hyps, "autotuned_shapes": shapes, **res,
            "fixed_S4096": {"autotuned_shapes": fixed_shapes, **res_f}}
    print(json.dumps(line), flush=True)


def _batch_windows(wl, S, iters, tune_hyps):
    """The windows of `wl` as library windows: each window's hypothesis count
    autotuned (tuning.autotune_hyps, from S/8, S/4, S/2 and S) or fixed at S,
    then its dense-scoring tile shape (voldor_autotune). Tuning is not timed."""
    from paper_2104_06789_gb300 import tuning, voldor
    wins, shapes, hyps = [], {}, {}
    for i, (b, T) in enumerate(wl):
        flows = np.ascontiguousarray(b.flows[:T].astype(np.float16))
        p = voldor.default_params(hyps_per_frame=S, inv_depth_min=b.inv_depth_range[0],
                                  inv_depth_max=b.inv_depth_range[1], window_id=i)
        if tune_hyps:
            s_win, _, _ = tuning.autotune_hyps(flows, b.K, p, b.poses[0], iters=iters)
            p.hyps_per_frame, p.groups_per_frame = s_win, 4 * s_win
        hyps[str(p.hyps_per_frame)] = hyps.get(str(p.hyps_per_frame), 0) + 1
        g = voldor.Window(flows, b.K, p)
        g.bootstrap(b.poses[0])
        hpt, ch, _ = g.autotune()
        shapes[f"{hpt}x{ch}"] = shapes.get(f"{hpt}x{ch}", 0) + 1
        wins.append((g, b, T))
    return wins, shapes, dict(sorted(hyps.items(), key=lambda kv: int(kv[0])))


def _batch_measure(wins, iters, pair_rate, warmup, steps):
    """One CUDA graph over `wins`: windows/s from the median batch wall time,
    per-window latency p50/p99 from the graph's own events, the same windows
    one after another (em_step each), the dense-scoring pairs (every window's
    scoring log) over `pair_rate` as the scoring-only lower bound, and the
    median over windows of the mean translation error. Destroys the windows."""
    import torch

    from paper_2104_06789_gb300 import voldor
    stream = torch.cuda.Stream()
    batch = voldor.Batch([g for g, _, _ in wins], iters)
    lat, walls = [], []
    for rep in range(warmup + steps):
        for g, b, _ in wins:
            g.bootstrap(b.poses[0])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        l = batch.run(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep >= warmup:
            lat.extend(l.tolist())
            walls.append(e0.elapsed_time(e1))
    batch.destroy()
    seq = []
    for _ in range(2):
        for g, b, _ in wins:
            g.bootstrap(b.poses[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g, _, _ in wins:
            g.em_step(iters)
        torch.cuda.synchronize()
        seq.append((time.perf_counter() - t0) * 1e3)
    pairs = 0.0
    for g, b, _ in wins:
        g.enable_timing(True)
        g.bootstrap(b.poses[0])
        g.em_step(iters)
        pairs += float(g.get_score_times()[1].sum())
        g.enable_timing(False)
    errs = []
    for g, b, T in wins:
        P, _, _ = g.get_pose_depth_rigidness(depth=False, rigidness=False)
        errs.append(float(np.mean(np.linalg.norm(P[:, :3, 3] - b.poses[:T, :3, 3], axis=1))))
        g.destroy()
    wall = float(np.median(walls))
    n = len(wins)
    units = sum(b.W * b.H * T * iters for _, b, T in wins)
    return {"windows_per_s": n / (wall / 1e3), "ms_per_batch": wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "mpixel_frame_per_s": units / (wall / 1e3) / 1e6,
            "sequential_ms": float(np.median(seq)), "speedup_vs_sequential": float(np.median(seq)) / wall,
            "scoring_pairs": pairs, "scoring_bound_ms": pairs / pair_rate * 1e3 if pair_rate else None,
            "scoring_bound_frac": (pairs / pair_rate * 1e3) / wall if pair_rate else None,
            "median_translation_error_m": float(np.median(errs))}


def batch_summary(iters, pair_rate, warmup=2, steps=3, n=64, S=4096):
    """Config 4 inside the default run: n windows of the mixed workload
    (batch_workload) in one CUDA graph, each window's hypothesis count and
    dense-scoring tile shape autotuned; beside it the same windows at a fixed
    S = 4096 with autotuned tile shapes. For each: windows/s, per-window
    latency p50/p99, the windows one after another, and the time the dense
    scoring alone needs at the driving window's measured pair rate (full-GPU
    occupancy), a lower bound for any batching of these windows with this
    scoring kernel."""
    from paper_2104_06789_gb300 import tuning
    wl = batch_workload(n)
    fixed, fixed_shapes, _ = _batch_windows(wl, S, iters, tune_hyps=False)
    res_fixed = _batch_measure(fixed, iters, pair_rate, warmup, steps)
    tuned, shapes, hyps = _batch_windows(wl, S, iters, tune_hyps=True)
    res = _batch_measure(tuned, iters, pair_rate, warmup, steps)
    return {"workload": f"{n} windows, resolutions uniform over 320x240 / 640x480 / 1242x375, T uniform in [3, 8]",
            "hyps_per_frame": f"autotuned per window from {sorted(tuning.default_candidates(S) + [S])}",
            "autotuned_hyps": hyps, "tile_shape": "autotuned per window", "shapes": shapes, "em_iters": iters,
            **res, "fixed_S4096": {"shapes": fixed_shapes, **res_fixed}}


WEIGHTS = os.path.join(ROOT, "paper_2104_06789_gb300", "weights", "proposal_handheld_1242x375_T8.npy")


def learned_summary(iters, heldout=16, S=4096):
    """The metric's second half inside the default run: the proposal network
    (weights trained on 2000 handheld windows at 1242x375, T = 8 by
    `bench.py --learned 2000`), evaluated on held-out windows: iterations and
    wall time (bootstrap + EM iterations, CUDA events) until the median pose
    error reaches the plain EM's after `iters` iterations (within 1 %)."""
    from paper_2104_06789_gb300 import learned, voldor
    if not os.path.exists(WEIGHTS):
        return {"unavailable": "trained weights not found"}
    net = voldor.Net(learned.SCENE["T"], np.load(WEIGHTS))
    held = learned.build_dataset([learned.HELDOUT_SEED0 + i for i in range(heldout)], S=S, label_iters=0,
                                 workers=max(1, min(heldout, (os.cpu_count() or 2) - 1)))
    res = learned.compare(net, held, S=S, max_iters=iters + 1, plain_iters=iters)
    net.destroy()
    out = {"workload": f"{heldout} held-out handheld windows at 1242x375 f=718 T=8 (scene seeds "
                       f"{learned.HELDOUT_SEED0}..{learned.HELDOUT_SEED0 + heldout - 1})",
           "hyps_per_frame": S, "target_median_err_m": res["median_target_err_m"],
           "plain": {"iters": iters, "ms": res["plain_ms"]}, "iteration_ms": res["iteration_ms"]}
    for m, name in (("learned_w", "learned_rigidness_prior"), ("learned", "learned_depth_and_rigidness")):
        k, ms = res[f"{m}_median_iters_to_target"], res[f"{m}_median_ms"]
        out[name] = {"iters": k, "ms": ms, "speedup": (res["plain_ms"] / ms) if ms else None,
                     "median_err_m": res[f"{m}_median_err_m"]}
    out["plain"]["median_err_m"] = res["plain_median_err_m"]
    return out


def measured_peaks():
    """The measured HBM copy bandwidth (GB/s) and bf16 GEMM rate
    (TFLOP/s, burst) of this GPU model, else the fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "fallback"


def run_net(args):
    """Proposal network forward throughput on B seeded random flow stacks of
    the learned workload's shape (1242x375, T = 8, FP16 flows; activations of
    238 MB per layer, larger than L2), and the training step at batch 2.
    Roofline of the forward pass as a whole (flow normalisation, input
    packing, six tcgen05 convolutions), layer by layer: HBM bytes per pixel =
    FP16 flows read twice (the per-frame magnitude sum, then the packing),
    2 x 32 B + packed input written and read 2 x 32 B + five 32-channel
    activations written and read 5 x 2 x 64 B + FP32 predictions 32 B = 800 B;
    FLOP per pixel = 2 x 9 x (2T x 32 + 4 x 32 x 32 + 32 x 2)."""
    import torch

    from paper_2104_06789_gb300 import build, learned, voldor
    torch.cuda.set_device(0)
    build.build()
    T, H, W, B = 8, 375, 1242, args.net
    rng = np.random.default_rng(0)
    flows = torch.from_numpy(rng.normal(0, 8, size=(B, T, H, W, 2)).astype(np.float16)).cuda()
    tgt = torch.from_numpy(np.stack([rng.normal(0, 0.5, size=(2, H, W)), rng.uniform(0, 1, size=(2, H, W))],
                                    -1).astype(np.float32)).cuda()
    net = voldor.Net(T, learned.init_weights(T))
    stream = torch.cuda.Stream()
    for _ in range(args.warmup):
        net.forward(flows, stream=stream)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(0) as clk:
        for e0, e1 in evs:
            e0.record(stream)
            net.forward(flows, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    f2, t2 = flows[:2].contiguous(), tgt
    for _ in range(args.warmup):
        net.train_step(f2, t2, 1e-4, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        net.train_step(f2, t2, 1e-4, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1) / args.steps
    net.destroy()
    hbm, bf16, src = measured_peaks()
    npx = B * H * W
    gbs = npx * 800 / (ms * 1e-3) / 1e9
    tflops = npx * 2 * 9 * (2 * T * 32 + 4 * 32 * 32 + 32 * 2) / (ms * 1e-3) / 1e12
    line = {"metric": "proposal network forward, images/s at 1242x375 T=8", "value": B / (ms * 1e-3),
            "unit": "images/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "dtype": "bf16", "data": "synthetic (seeded normal flows)",
            "config": {"workload": "proposal_net_1242x375_T8", "images": B, "flows": "fp16",
                       "l2": "activations 238 MB per layer, larger than L2"},
            "roofline": {"kernel": "forward pass (normalisation, packing, 6 x k_conv_tc)", "bound": "hbm", "achieved": gbs,
                         "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
                         "tensor_tflops": tflops, "tensor_frac": tflops / bf16, "peak_source": src},
            "train_step_batch2_ms": train_ms, "train_mpix_per_s": 2 * H * W / (train_ms * 1e-3) / 1e6,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_learned(args):
    """Plain vs learned initialisation: generate and label the training
    windows, train the proposal network with the library's kernels, compare
    the pose error per EM iteration and the time to the plain EM's error on
    held-out windows."""
    import torch

    from paper_2104_06789_gb300 import build, learned, voldor
    workers = args.workers or max(1, (os.cpu_count() or 2) - 1)
    log = lambda m: print(f"[learned] {m}", file=sys.stderr, flush=True)
    S = 4096
    torch.cuda.set_device(0)
    build.build()
    t0 = time.time()
    train_seeds = [learned.TRAIN_SEED0 + i for i in range(args.learned)]
    held_seeds = [learned.HELDOUT_SEED0 + i for i in range(args.heldout)]
    T = learned.SCENE["T"]
    t_data = t_train = 0.0
    losses = np.zeros(1)
    pix_per_step = 2 * learned.SCENE["W"] * learned.SCENE["H"]
    if args.weights:
        net = voldor.Net(T, np.load(args.weights))
        log(f"weights from {args.weights}: no training")
    else:
        ds = learned.build_dataset(train_seeds, S=S, label_iters=8, workers=workers, log=log)
        t_data = time.time() - t0
        log(f"training set: {ds.n} windows in {t_data:.0f} s")
        net = voldor.Net(T, learned.init_weights(T, seed=0))
        t1 = time.time()
        losses = learned.train(net, ds, args.train_steps, batch=2, lr=1e-3, log=log)
        torch.cuda.synchronize()
        t_train = time.time() - t1
        if args.save_weights:
            np.save(args.save_weights, net.get_weights())
        del ds
    held = learned.build_dataset(held_seeds, S=S, label_iters=0, workers=workers, log=log)
    res = learned.compare(net, held, S=S, max_iters=8, plain_iters=args.iters)
    # value: the faster learned initialisation's time to the plain EM's median error after
    # args.iters iterations (null if neither reaches it within 8 iterations)
    cands = [(res[f"{m}_median_ms"], m) for m in ("learned", "learned_w") if res[f"{m}_median_ms"] is not None]
    best = min(cands) if cands else (None, None)
    line = {"metric": "wall time to the plain EM's median pose error (bootstrap + EM iterations), learned init",
            "value": best[0], "value_variant": best[1], "plain_ms_same_metric": res["plain_ms"],
            "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "data": "synthetic", "dtype": "bf16 net, f32/f64 EM",
            "config": {"workload": "handheld scenes at 1242x375 f=718 T=8", "train_windows": len(train_seeds),
                       "heldout_windows": len(held_seeds), "hyps_per_frame": S, "train_steps": args.train_steps,
                       "batch": 2, "label_iters": 8},
            "train_s": t_train,
            "train_mpix_per_s": pix_per_step * args.train_steps / t_train / 1e6 if t_train else None,
            "loss_first_last": [float(losses[:50].mean()), float(losses[-50:].mean())],
            "data_s": t_data, **res}
    print(json.dumps(line), flush=True)
    net.destroy()


def run_probe_sfu():
    """The SFU probe alone (one launch per op after its warm-up), for an ncu
    capture of the probe kernel's pipe counters beside its own figures."""
    import torch

    from paper_2104_06789_gb300 import build, voldor
    torch.cuda.set_device(0)
    build.build()
    out = {}
    for op, name in enumerate(("ex2", "lg2", "rcp")):
        r, f = voldor.probe_sfu_rate(op, with_clock=True)
        out[name] = {"results_per_sm_clock": r, "sm_mhz": f}
    print(json.dumps({"sfu_probe": out}), flush=True)


def main():
    args = parse_args()
    if args.probe_sfu:
        run_probe_sfu()
    elif args.net:
        run_net(args)
    elif args.learned:
        run_learned(args)
    elif args.batch:
        run_batch(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
