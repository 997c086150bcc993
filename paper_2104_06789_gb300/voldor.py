"""Python binding of libvoldor.so (include/voldor.h): argument marshalling only.

Every step of the inference runs in the library's CUDA kernels. Host arrays
are numpy; device arrays may be torch CUDA tensors (their data pointers are
passed through). There is no fallback: if the library or a GPU is missing,
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvoldor.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_BOOTSTRAPPED, ERR_DEGENERATE, ERR_TIMEOUT, ERR_INTERNAL = range(8)
FLOW_F32, FLOW_F16 = 0, 1
LEARNED_DEPTH, LEARNED_RIGIDNESS = 1, 2
CRITERION_MIE, CRITERION_MLE = 0, 1
RESIDUAL_FISK, RESIDUAL_GAUSSIAN = 0, 1
BOOT_GIVEN_POSE, BOOT_EPIPOLAR = 0, 2
(BUF_SMOOTHED, BUF_LABELS, BUF_HYPS, BUF_HYP_INFO, BUF_HYP_WEIGHT, BUF_SCORES, BUF_POSE_INFO,
 BUF_DEPTH_SAMPLES, BUF_HYPS_F32, BUF_EPI_E, BUF_EPI_MEDIANS, BUF_EPI_VALID, BUF_EPI_INFO,
 BUF_EPI_REFINED) = range(14)
EPI_MAX_SAMPLES = 4096


class VoldorError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class Params(C.Structure):
    _fields_ = [
        ("a1", C.c_double), ("a2", C.c_double), ("b1", C.c_double), ("b2", C.c_double),
        ("lambda_", C.c_double), ("gamma", C.c_double),
        ("sigma_t", C.c_double), ("sigma_r", C.c_double),
        ("inv_depth_min", C.c_double), ("inv_depth_max", C.c_double),
        ("x_min", C.c_double), ("x_max", C.c_double), ("beta_min", C.c_double),
        ("ms_tol", C.c_double),
        ("hyps_per_frame", C.c_int), ("groups_per_frame", C.c_int),
        ("ms_max_iter", C.c_int), ("criterion", C.c_int), ("residual", C.c_int),
        ("seed", C.c_uint64), ("window_id", C.c_uint64),
    ]


class Intrinsics(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double)]


_lib = None


def lib():
    """Loads libvoldor.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2104_06789_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
        P = C.POINTER
        sig = {
            "voldor_default_params": (None, [P(Params)]),
            "voldor_status_string": (C.c_char_p, [i]),
            "voldor_init_window": (i, [P(vp), i, i, i, P(Intrinsics), P(Params), vp, i, i, vp]),
            "voldor_set_flows": (i, [vp, vp, i]),
            "voldor_bootstrap": (i, [vp, i, P(d)]),
            "voldor_em_step": (i, [vp, i]),
            "voldor_get_pose_depth_rigidness": (i, [vp, P(d), P(C.c_float), P(C.c_float)]),
            "voldor_destroy": (None, [vp]),
            "voldor_set_state": (i, [vp, P(d), P(C.c_float), P(C.c_float), i]),
            "voldor_pose_update": (i, [vp, i, i]),
            "voldor_score_hypotheses": (i, [vp, i, i, P(d), P(d), P(d)]),
            "voldor_rigidness_smooth": (i, [vp, i]),
            "voldor_depth_update": (i, [vp, i]),
            "voldor_rigidness_update": (i, [vp]),
            "voldor_get_buffer": (i, [vp, i, vp, sz]),
            "voldor_set_buffer": (i, [vp, i, vp, sz]),
            "voldor_enable_timing": (i, [vp, i]),
            "voldor_get_score_times": (i, [vp, P(C.c_float), P(C.c_longlong), P(C.c_longlong), i, P(i)]),
            "voldor_kernel_launches": (C.c_longlong, [vp]),
            "voldor_last_error_string": (C.c_char_p, [vp]),
            "voldor_device_bytes": (sz, [vp]),
            "voldor_score_records_noalloc": (i, [vp, i, vp, i, d, d, vp, vp]),
            "voldor_probe_sfu_rate": (i, [i, P(d), P(d)]),
            "voldor_probe_bounded_wait": (i, [C.c_longlong, P(C.c_longlong)]),
            "voldor_autotune": (i, [vp, P(i), P(i), P(C.c_float)]),
            "voldor_set_score_shape": (i, [vp, i, i]),
            "voldor_batch_create": (i, [P(vp), i, i, P(vp)]),
            "voldor_batch_run": (i, [vp, vp, P(C.c_float)]),
            "voldor_batch_destroy": (None, [vp]),
            "voldor_em_batch": (i, [P(vp), i, i]),
            "voldor_net_num_params": (sz, [i]),
            "voldor_net_create": (i, [i, P(vp)]),
            "voldor_net_destroy": (None, [vp]),
            "voldor_net_set_weights": (i, [vp, P(C.c_float), sz]),
            "voldor_net_get_weights": (i, [vp, P(C.c_float), sz]),
            "voldor_net_get_grads": (i, [vp, P(C.c_float), sz]),
            "voldor_net_forward": (i, [vp, vp, i, i, i, i, vp, vp]),
            "voldor_net_train_step": (i, [vp, vp, i, vp, i, i, i, C.c_float, C.c_float, P(C.c_float), vp]),
            "voldor_bootstrap_learned": (i, [vp, P(d), vp, i]),
            "voldor_bootstrap_epipolar": (i, [vp, i, d, P(d)]),
            "voldor_ground_scale": (i, [vp, d, d, i, P(d)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(s):
    return lib().voldor_status_string(int(s)).decode()


def _check(st, where, allow=(), handle=None):
    if st != OK and st not in allow:
        if st == ERR_CUDA and handle:
            where = f"{where} [{lib().voldor_last_error_string(handle).decode()}]"
        raise VoldorError(st, where)
    return st


def _require_shape(name, a, shape):
    # the C calls read exactly this many elements from the pointer they get
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(a.shape)}")


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


def default_params(**overrides) -> Params:
    """The library's defaults with overrides; the group budget follows S
    (4 S) unless it is given."""
    p = Params()
    lib().voldor_default_params(C.byref(p))
    if "hyps_per_frame" in overrides and "groups_per_frame" not in overrides:
        overrides = dict(overrides, groups_per_frame=4 * int(overrides["hyps_per_frame"]))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _flow_arg(flows):
    """(pointer, on_device, dtype, keepalive) of a numpy array or torch tensor."""
    if hasattr(flows, "data_ptr") and hasattr(flows, "is_cuda"):
        import torch
        t = flows.contiguous()
        dt = {torch.float32: FLOW_F32, torch.float16: FLOW_F16}[t.dtype]
        if t.is_cuda:
            return C.c_void_p(t.data_ptr()), 1, dt, t
        a = t.numpy()
    else:
        a = np.asarray(flows)
    if a.dtype == np.float16:
        a = np.ascontiguousarray(a)
        return C.c_void_p(a.ctypes.data), 0, FLOW_F16, a
    a = np.ascontiguousarray(a, dtype=np.float32)
    return C.c_void_p(a.ctypes.data), 0, FLOW_F32, a


class Window:
    """One VOLDOR window (a voldor_ctx)."""

    def __init__(self, flows, K, params: Params | None = None, stream=None):
        shape = tuple(flows.shape)
        assert len(shape) == 4 and shape[3] == 2, "flows must be [T][H][W][2]"
        self.T, self.H, self.W = shape[:3]
        ptr, on_dev, dt, keep = _flow_arg(flows)
        self.flow_dtype = dt
        self.params = params if params is not None else default_params()
        self.K = Intrinsics(*[float(v) for v in K])
        h = C.c_void_p()
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        self._stream = stream
        _check(lib().voldor_init_window(C.byref(h), self.W, self.H, self.T, C.byref(self.K), C.byref(self.params),
                                        ptr, dt, on_dev, C.c_void_p(st)), "voldor_init_window")
        self._h = h

    # -- lifetime -----------------------------------------------------------
    def destroy(self):
        if getattr(self, "_h", None):
            lib().voldor_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    # -- main calls -------------------------------------------------------------
    def set_flows(self, flows):
        ptr, on_dev, dt, keep = _flow_arg(flows)
        assert dt == self.flow_dtype
        _check(lib().voldor_set_flows(self._h, ptr, on_dev), "voldor_set_flows", handle=self._h)

    def bootstrap(self, T1):
        T1, p = _f64(T1)
        _require_shape("T1", T1, (4, 4))
        _check(lib().voldor_bootstrap(self._h, BOOT_GIVEN_POSE, p), "voldor_bootstrap", handle=self._h)

    def bootstrap_epipolar(self, n_samples=512, baseline=1.0):
        """T_1 by least median of squares on X_1, then the bootstrap; returns T_1."""
        T1 = np.zeros(16)
        _check(lib().voldor_bootstrap_epipolar(self._h, int(n_samples), float(baseline),
                                               T1.ctypes.data_as(C.POINTER(C.c_double))),
               "voldor_bootstrap_epipolar", handle=self._h)
        self._epi_M = int(n_samples)
        return T1.reshape(4, 4)

    def ground_scale(self, camera_height, max_tilt_deg=10.0, apply=False):
        """Scale that puts the ground plane of the current depth at
        camera_height below the camera (applied to the depth and the
        translations if apply)."""
        s = C.c_double(0.0)
        _check(lib().voldor_ground_scale(self._h, float(camera_height), float(np.deg2rad(max_tilt_deg)),
                                         1 if apply else 0, C.byref(s)), "voldor_ground_scale", handle=self._h)
        return s.value

    def epipolar_results(self):
        """Per-sample essential matrices, medians and validity, and the
        chosen sample / candidate, valid-pixel and inlier counts, cheirality
        counts and the refined E, U, V of the last epipolar bootstrap."""
        M = self._epi_M
        E = self.get_buffer(BUF_EPI_E, (M, 3, 3), np.float64)
        med = self.get_buffer(BUF_EPI_MEDIANS, (M,), np.float32)
        valid = self.get_buffer(BUF_EPI_VALID, (M,), np.int32)
        info = self.get_buffer(BUF_EPI_INFO, (8,), np.int64)
        ref = self.get_buffer(BUF_EPI_REFINED, (3, 3, 3), np.float64)
        return dict(E=E, medians=med, valid=valid > 0, why=valid, chosen=int(info[0]), candidate=int(info[1]),
                    n_valid=int(info[2]), n_inliers=int(info[3]), counts=info[4:].copy(),
                    E_refined=ref[0], U=ref[1], V=ref[2])

    def em_step(self, n_iters, allow_degenerate=True):
        allow = (ERR_DEGENERATE,) if allow_degenerate else ()
        return _check(lib().voldor_em_step(self._h, int(n_iters)), "voldor_em_step", allow, handle=self._h)

    def get_pose_depth_rigidness(self, poses=True, depth=True, rigidness=True):
        P = np.zeros((self.T, 4, 4)) if poses else None
        D = np.zeros((self.H, self.W), np.float32) if depth else None
        Wm = np.zeros((self.T, self.H, self.W), np.float32) if rigidness else None
        nul = lambda a, t: a.ctypes.data_as(C.POINTER(t)) if a is not None else None
        _check(lib().voldor_get_pose_depth_rigidness(self._h, nul(P, C.c_double), nul(D, C.c_float),
                                                     nul(Wm, C.c_float)), "voldor_get_pose_depth_rigidness", handle=self._h)
        return P, D, Wm

    # -- stage calls ------------------------------------------------------------
    def set_state(self, poses=None, depth=None, rigidness=None, iteration=0):
        keep = []

        def arg(a, conv, name, shape):
            if a is None:
                return None
            a, p = conv(a)
            _require_shape(name, a, shape)
            keep.append(a)
            return p

        _check(lib().voldor_set_state(self._h, arg(poses, _f64, "poses", (self.T, 4, 4)),
                                      arg(depth, _f32, "depth", (self.H, self.W)),
                                      arg(rigidness, _f32, "rigidness", (self.T, self.H, self.W)),
                                      int(iteration)), "voldor_set_state", handle=self._h)

    def pose_update(self, k, t):
        return _check(lib().voldor_pose_update(self._h, int(k), int(t)), "voldor_pose_update", (ERR_DEGENERATE,), handle=self._h)

    def score_hypotheses(self, t, R, tv):
        R, pR = _f64(R)
        tv, pt = _f64(tv)
        n = R.shape[0]
        _require_shape("R", R, (n, 3, 3))
        _require_shape("tv", tv, (n, 3))
        L = np.zeros(n)
        _check(lib().voldor_score_hypotheses(self._h, int(t), n, pR, pt, L.ctypes.data_as(C.POINTER(C.c_double))),
               "voldor_score_hypotheses", handle=self._h)
        return L

    def rigidness_smooth(self, k):
        _check(lib().voldor_rigidness_smooth(self._h, int(k)), "voldor_rigidness_smooth", handle=self._h)

    def depth_update(self, k):
        _check(lib().voldor_depth_update(self._h, int(k)), "voldor_depth_update", handle=self._h)

    def rigidness_update(self):
        _check(lib().voldor_rigidness_update(self._h), "voldor_rigidness_update", handle=self._h)

    def get_buffer(self, which, shape, dtype):
        out = np.zeros(shape, dtype=dtype)
        _check(lib().voldor_get_buffer(self._h, which, C.c_void_p(out.ctypes.data), out.nbytes), "voldor_get_buffer", handle=self._h)
        return out

    def set_buffer(self, which, arr):
        arr = np.ascontiguousarray(arr)
        _check(lib().voldor_set_buffer(self._h, which, C.c_void_p(arr.ctypes.data), arr.nbytes), "voldor_set_buffer", handle=self._h)

    def enable_timing(self, on=True):
        _check(lib().voldor_enable_timing(self._h, int(bool(on))), "voldor_enable_timing", handle=self._h)

    def get_score_times(self, max_n=1024, with_hyps=False):
        """(ms per scoring launch, pairs per launch[, hypotheses per launch])
        of the last timed em_step."""
        ms = np.zeros(max_n, np.float32)
        pairs = np.zeros(max_n, np.int64)
        hyps = np.zeros(max_n, np.int64)
        n = C.c_int(0)
        _check(lib().voldor_get_score_times(self._h, ms.ctypes.data_as(C.POINTER(C.c_float)),
                                            pairs.ctypes.data_as(C.POINTER(C.c_longlong)),
                                            hyps.ctypes.data_as(C.POINTER(C.c_longlong)), max_n, C.byref(n)),
               "voldor_get_score_times", handle=self._h)
        m = min(n.value, max_n)
        return (ms[:m], pairs[:m], hyps[:m]) if with_hyps else (ms[:m], pairs[:m])

    def kernel_launches(self):
        return int(lib().voldor_kernel_launches(self._h))

    def device_bytes(self):
        return lib().voldor_device_bytes(self._h)

    def autotune(self):
        """(hypotheses per thread, pixel chunks, best ms) chosen for this window."""
        hpt, ch, ms = C.c_int(0), C.c_int(0), C.c_float(0)
        _check(lib().voldor_autotune(self._h, C.byref(hpt), C.byref(ch), C.byref(ms)), "voldor_autotune",
               handle=self._h)
        return hpt.value, ch.value, ms.value

    def set_score_shape(self, hyps_per_thread, chunks):
        _check(lib().voldor_set_score_shape(self._h, int(hyps_per_thread), int(chunks)), "voldor_set_score_shape",
               handle=self._h)

    # -- convenience readers of the stage buffers -----------------------------------
    def hypotheses(self):
        S = self.params.hyps_per_frame
        info = self.get_buffer(BUF_POSE_INFO, (4,), np.int32)
        n = int(info[0])
        hyps = self.get_buffer(BUF_HYPS, (S, 12), np.float64)[:n]
        hinfo = self.get_buffer(BUF_HYP_INFO, (S, 2), np.int64)[:n]
        w = self.get_buffer(BUF_HYP_WEIGHT, (S,), np.float64)[:n]
        L = self.get_buffer(BUF_SCORES, (S,), np.float64)[:n]
        return dict(R=hyps[:, :9].reshape(-1, 3, 3), t=hyps[:, 9:], group=hinfo[:, 0], slot=hinfo[:, 1],
                    weight=w, L=L, seed=int(info[1]), ms_iters=int(info[2]), degenerate=int(info[3]))


def score_records_noalloc(records, hyps, L, xs_min, xs_max, stream=None):
    """Allocation-free dense scoring (voldor_score_records_noalloc).

    records: CUDA float32 tensor [n_pix, 12]; hyps: CUDA float32 tensor
    [n_hyps, 12]; L: CUDA float64 tensor [n_hyps], written asynchronously on
    `stream`. Allocates no device memory.
    """
    import torch
    for name, x, dt, width in (("records", records, torch.float32, 12), ("hyps", hyps, torch.float32, 12),
                               ("L", L, torch.float64, None)):
        if not x.is_cuda or x.dtype != dt or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor")
        if width is not None and (x.dim() != 2 or x.shape[1] != width):
            raise ValueError(f"{name} must have shape [n, {width}]")
    if L.numel() < hyps.shape[0]:
        raise ValueError("L needs one entry per hypothesis")
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    _check(lib().voldor_score_records_noalloc(C.c_void_p(records.data_ptr()), int(records.shape[0]),
                                              C.c_void_p(hyps.data_ptr()), int(hyps.shape[0]), float(xs_min),
                                              float(xs_max), C.c_void_p(L.data_ptr()), C.c_void_p(st)),
           "voldor_score_records_noalloc")


def probe_sfu_rate(op, with_clock=False):
    """SFU results per SM clock of the current GPU: op 0 exp2, 1 log2, 2 rcp
    (with_clock: also the SM clock in MHz measured during the probe)."""
    v, f = C.c_double(0.0), C.c_double(0.0)
    _check(lib().voldor_probe_sfu_rate(int(op), C.byref(v), C.byref(f)), "voldor_probe_sfu_rate")
    return (v.value, f.value) if with_clock else v.value


def probe_bounded_wait(polls):
    """(status, SM cycles) of the bounded-wait expiry probe: ERR_TIMEOUT is the
    expected status (nothing completes the phase the probe waits on)."""
    cyc = C.c_longlong(0)
    st = lib().voldor_probe_bounded_wait(int(polls), C.byref(cyc))
    return st, cyc.value


class Batch:
    """Windows run together as one CUDA graph (voldor_batch_*)."""

    def __init__(self, windows, n_iters):
        self.windows = list(windows)
        arr = (C.c_void_p * len(self.windows))(*[w._h for w in self.windows])
        h = C.c_void_p()
        _check(lib().voldor_batch_create(arr, len(self.windows), int(n_iters), C.byref(h)), "voldor_batch_create")
        self._h = h

    def run(self, stream=None, latency=True):
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        lat = np.zeros(len(self.windows), np.float32)
        _check(lib().voldor_batch_run(self._h, C.c_void_p(st), lat.ctypes.data_as(C.POINTER(C.c_float)) if latency
                                      else None), "voldor_batch_run", (ERR_DEGENERATE,))
        return lat

    def destroy(self):
        if getattr(self, "_h", None):
            lib().voldor_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def em_batch(windows, n_iters):
    arr = (C.c_void_p * len(windows))(*[w._h for w in windows])
    return _check(lib().voldor_em_batch(arr, len(windows), int(n_iters)), "voldor_em_batch", (ERR_DEGENERATE,))


class Net:
    """The learned proposal network (voldor_net_*). Device arrays are torch
    CUDA tensors: flows [B][T][H][W][2] (float16 or float32), targets
    [B][H][W][2] float32, predictions [B][H][W][8] float32."""

    def __init__(self, T, weights=None):
        self.T = int(T)
        self.n_params = int(lib().voldor_net_num_params(self.T))
        h = C.c_void_p()
        _check(lib().voldor_net_create(self.T, C.byref(h)), "voldor_net_create")
        self._h = h
        if weights is not None:
            self.set_weights(weights)

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(lib().voldor_net_set_weights(self._h, w.ctypes.data_as(C.POINTER(C.c_float)), w.size),
               "voldor_net_set_weights")

    def get_weights(self):
        w = np.zeros(self.n_params, np.float32)
        _check(lib().voldor_net_get_weights(self._h, w.ctypes.data_as(C.POINTER(C.c_float)), w.size),
               "voldor_net_get_weights")
        return w

    def get_grads(self):
        g = np.zeros(self.n_params, np.float32)
        _check(lib().voldor_net_get_grads(self._h, g.ctypes.data_as(C.POINTER(C.c_float)), g.size),
               "voldor_net_get_grads")
        return g

    @staticmethod
    def _flow_dtype(t):
        import torch
        return {torch.float16: FLOW_F16, torch.float32: FLOW_F32}[t.dtype]

    def forward(self, flows, stream=None):
        import torch
        B, T, H, W = flows.shape[:4]
        out = torch.empty((B, H, W, 8), dtype=torch.float32, device=flows.device)
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        _check(lib().voldor_net_forward(self._h, C.c_void_p(flows.data_ptr()), self._flow_dtype(flows), B, H, W,
                                        C.c_void_p(out.data_ptr()), C.c_void_p(st)), "voldor_net_forward")
        return out

    def train_step(self, flows, target, lr, lam_r=1.0, stream=None):
        B, T, H, W = flows.shape[:4]
        loss = C.c_float(0)
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        _check(lib().voldor_net_train_step(self._h, C.c_void_p(flows.data_ptr()), self._flow_dtype(flows),
                                           C.c_void_p(target.data_ptr()), B, H, W, float(lr), float(lam_r),
                                           C.byref(loss), C.c_void_p(st)), "voldor_net_train_step")
        return loss.value

    def bootstrap(self, window, T1, depth=True, rigidness=True):
        T1, p = _f64(T1)
        flags = (LEARNED_DEPTH if depth else 0) | (LEARNED_RIGIDNESS if rigidness else 0)
        _check(lib().voldor_bootstrap_learned(window._h, p, self._h, flags), "voldor_bootstrap_learned",
               handle=window._h)

    def destroy(self):
        if getattr(self, "_h", None):
            lib().voldor_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def init_window(flows, K, params=None, stream=None) -> Window:
    return Window(flows, K, params, stream)
