"""ctypes loader of the FP64 VOLDOR oracle (``voldor_oracle.cpp``).

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` import this package. The product path
(``paper_2104_06789_gb300``) never imports it, and the two share no code.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "voldor_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (IEEE FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", _LIB, _SRC]
        subprocess.run(cmd, check=True)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("a1", C.c_double), ("a2", C.c_double), ("b1", C.c_double), ("b2", C.c_double),
        ("lambda_", C.c_double), ("gamma", C.c_double),
        ("sigma_t", C.c_double), ("sigma_r", C.c_double),
        ("inv_depth_min", C.c_double), ("inv_depth_max", C.c_double),
        ("x_min", C.c_double), ("x_max", C.c_double), ("beta_min", C.c_double),
        ("ms_tol", C.c_double),
        ("hyps_per_frame", C.c_int), ("groups_per_frame", C.c_int),
        ("ms_max_iter", C.c_int), ("pad_", C.c_int),
        ("seed", C.c_uint64), ("window_id", C.c_uint64),
    ]


class Window(C.Structure):
    _fields_ = [
        ("width", C.c_int), ("height", C.c_int), ("T", C.c_int), ("pad_", C.c_int),
        ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
        ("p", Params),
        ("flows", C.POINTER(C.c_double)), ("theta", C.POINTER(C.c_double)),
        ("wmap", C.POINTER(C.c_double)), ("poses", C.POINTER(C.c_double)),
    ]


# The paper's hyper-parameters (Sec. 6.1) and the readings' numerical guards.
PAPER_DEFAULTS = dict(a1=0.01, a2=0.09, b1=-0.0022, b2=1.0, lambda_=0.15, gamma=0.9,
                      sigma_t=0.1, sigma_r=0.004, x_min=1e-6, x_max=1e12, beta_min=0.05,
                      ms_tol=1e-10, ms_max_iter=100)

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, u64 = C.c_double, C.c_int, C.c_uint64
        P = C.POINTER
        W = P(Window)
        sig = {
            "or_philox4x64_10": (None, [P(u64), P(u64), P(u64)]),
            "or_fisk_logpdf": (d, [d, d, d]),
            "or_fisk_params": (None, [P(Params), d, P(d), P(d)]),
            "or_frame_ell": (d, [W, i, i, d, P(i)]),
            "or_frame_eval": (i, [W, i, i, d, P(d)]),
            "or_bilinear": (i, [W, i, d, d, P(d)]),
            "or_bootstrap": (None, [W, P(d)]),
            "or_p3p": (i, [P(d), P(d), P(d), P(d), P(d)]),
            "or_draw_group": (i, [W, i, i, C.c_int64, P(C.c_int64)]),
            "or_collect_hypotheses": (i, [W, i, i, P(d), P(d), P(d), P(C.c_int64), P(i)]),
            "or_score_hypotheses": (None, [W, i, i, P(d), P(d), P(d)]),
            "or_se3_exp": (None, [P(d), P(d), P(d)]),
            "or_se3_log": (None, [P(d), P(d), P(d)]),
            "or_meanshift": (i, [P(d), P(d), i, i, d, d, i, d, P(d)]),
            "or_pose_update": (i, [W, i, i, P(i), P(d), P(i), P(i)]),
            "or_emissions": (None, [W, P(d)]),
            "or_forward_backward": (None, [P(d), i, d, P(d)]),
            "or_smooth": (None, [W, i, P(d), P(d)]),
            "or_mie_score": (d, [W, P(d), i, d]),
            "or_depth_sample": (d, [W, i, C.c_int64]),
            "or_mie_sweep": (None, [W, i, P(d), P(C.c_ubyte)]),
            "or_rigidness": (None, [W]),
            "or_em_iteration": (i, [W, i]),
            "or_run": (i, [W, i, i]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def ptr(a: np.ndarray, ctype):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(ctype))


class OracleWindow:
    """FP64 window state owned by numpy arrays, viewed by the C oracle."""

    def __init__(self, flows, K, S=256, G=None, seed=0, window_id=0,
                 inv_depth_min=1.0 / 40.0, inv_depth_max=1.0, **overrides):
        flows = np.ascontiguousarray(np.asarray(flows, dtype=np.float64))
        assert flows.ndim == 4 and flows.shape[3] == 2
        self.T, self.H, self.W = flows.shape[:3]
        self.flows = flows
        self.theta = np.zeros((self.H, self.W))
        self.wmap = np.ones((self.T, self.H, self.W))
        self.poses = np.tile(np.eye(4), (self.T, 1, 1)).astype(np.float64)
        prm = dict(PAPER_DEFAULTS)
        prm.update(inv_depth_min=inv_depth_min, inv_depth_max=inv_depth_max,
                   hyps_per_frame=S, groups_per_frame=2 * S if G is None else G,
                   seed=seed, window_id=window_id)
        prm.update(overrides)
        self.params = Params(**prm)
        fx, fy, cx, cy = K
        self.K = (float(fx), float(fy), float(cx), float(cy))
        self._win = Window(self.W, self.H, self.T, 0, fx, fy, cx, cy, self.params,
                           _dp(self.flows), _dp(self.theta), _dp(self.wmap), _dp(self.poses))

    @property
    def ref(self):
        # refresh pointers in case arrays were replaced
        w = self._win
        w.theta = _dp(self.theta)
        w.wmap = _dp(self.wmap)
        w.poses = _dp(self.poses)
        w.flows = _dp(self.flows)
        w.p = self.params
        return C.byref(w)

    # -- thin wrappers -------------------------------------------------------
    def bootstrap(self, T1):
        T1 = np.ascontiguousarray(T1, dtype=np.float64)
        lib().or_bootstrap(self.ref, _dp(T1))

    def frame_eval(self, t, j, depth):
        out = np.zeros(12)
        v = lib().or_frame_eval(self.ref, t, j, depth, _dp(out))
        return v, out

    def collect_hypotheses(self, k, t):
        S = self.params.hyps_per_frame
        R = np.zeros((S, 3, 3)); tv = np.zeros((S, 3)); w = np.zeros(S)
        g = np.zeros(S, dtype=np.int64); s = np.zeros(S, dtype=np.int32)
        n = lib().or_collect_hypotheses(self.ref, k, t, _dp(R), _dp(tv), _dp(w),
                                        ptr(g, C.c_int64), ptr(s, C.c_int))
        return R[:n], tv[:n], w[:n], g[:n], s[:n]

    def score(self, t, R, tv):
        R = np.ascontiguousarray(R, dtype=np.float64)
        tv = np.ascontiguousarray(tv, dtype=np.float64)
        n = R.shape[0]
        L = np.zeros(n)
        lib().or_score_hypotheses(self.ref, t, n, _dp(R), _dp(tv), _dp(L))
        return L

    def pose_update(self, k, t):
        S = self.params.hyps_per_frame
        n = C.c_int(0); seed = C.c_int(0); its = C.c_int(0)
        L = np.zeros(S)
        st = lib().or_pose_update(self.ref, k, t, C.byref(n), _dp(L), C.byref(seed), C.byref(its))
        return st, n.value, L[:n.value], seed.value, its.value

    def emissions(self):
        out = np.zeros((self.T, self.H, self.W))
        lib().or_emissions(self.ref, _dp(out))
        return out

    def smooth(self, axis, emis):
        emis = np.ascontiguousarray(emis, dtype=np.float64)
        q = np.zeros_like(emis)
        lib().or_smooth(self.ref, axis, _dp(emis), _dp(q))
        return q

    def mie_sweep(self, k, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        labels = np.zeros((self.H, self.W), dtype=np.uint8)
        lib().or_mie_sweep(self.ref, k, _dp(q), ptr(labels, C.c_ubyte))
        return labels

    def mie_score(self, q, j, depth):
        q = np.ascontiguousarray(q, dtype=np.float64)
        return lib().or_mie_score(self.ref, _dp(q), j, depth)

    def depth_sample(self, k, j):
        return lib().or_depth_sample(self.ref, k, j)

    def rigidness(self):
        lib().or_rigidness(self.ref)

    def em_iteration(self, k):
        return lib().or_em_iteration(self.ref, k)

    def run(self, k0, n):
        return lib().or_run(self.ref, k0, n)


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64_10(ptr(c, C.c_uint64), ptr(k, C.c_uint64), ptr(out, C.c_uint64))
    return out


def fisk_logpdf(x, log_alpha, beta):
    return lib().or_fisk_logpdf(float(x), float(log_alpha), float(beta))


def p3p(P, b):
    P = np.ascontiguousarray(P, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    R = np.zeros((4, 3, 3)); t = np.zeros((4, 3)); s1 = np.zeros(4)
    n = lib().or_p3p(_dp(P), _dp(b), _dp(R), _dp(t), _dp(s1))
    return R[:n], t[:n], s1[:n]


def se3_exp(p):
    p = np.ascontiguousarray(p, dtype=np.float64)
    R = np.zeros((3, 3)); t = np.zeros(3)
    lib().or_se3_exp(_dp(p), _dp(R), _dp(t))
    return R, t


def se3_log(R, t):
    R = np.ascontiguousarray(R, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    p = np.zeros(6)
    lib().or_se3_log(_dp(R), _dp(t), _dp(p))
    return p


def meanshift(p, w, seed, sigma_t, sigma_r, max_iter=100, tol=1e-12):
    p = np.ascontiguousarray(p, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.zeros(6)
    it = lib().or_meanshift(_dp(p), _dp(w), p.shape[0], seed, sigma_t, sigma_r, max_iter, tol, _dp(x))
    return it, x


def forward_backward(w, gamma):
    w = np.ascontiguousarray(w, dtype=np.float64)
    q = np.zeros_like(w)
    lib().or_forward_backward(_dp(w), w.shape[0], gamma, _dp(q))
    return q
