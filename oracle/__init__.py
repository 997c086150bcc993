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
        ("ms_max_iter", C.c_int), ("criterion", C.c_int), ("residual", C.c_int),
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
            "or_gauss_logpdf": (d, [d, d]),
            "or_fisk_params": (None, [P(Params), d, P(d), P(d)]),
            "or_frame_ell": (d, [W, i, i, d, P(i)]),
            "or_frame_crit": (d, [W, i, i, d]),
            "or_frame_eval": (i, [W, i, i, d, P(d)]),
            "or_bilinear": (i, [W, i, d, d, P(d)]),
            "or_bootstrap": (None, [W, P(d)]),
            "or_p3p": (i, [P(d), P(d), P(d), P(d), P(d)]),
            "or_valid_pixels": (C.c_int64, [W, i, P(C.c_int64)]),
            "or_draw_group": (i, [W, i, i, C.c_int64, P(C.c_int64), C.c_int64, P(C.c_int64)]),
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
            "or_essential_8pt": (i, [P(d), P(d), P(d)]),
            "or_essential_project": (i, [P(d), P(d), P(d), P(d)]),
            "or_sampson": (d, [P(d), P(d), P(d)]),
            "or_essential_candidates": (None, [P(d), P(d), P(d), P(d)]),
            "or_epi_sample": (i, [W, i, P(d), P(C.c_int64)]),
            "or_epi_score": (d, [W, P(d)]),
            "or_epi_cheirality": (C.c_int64, [W, P(d), P(d)]),
            "or_epipolar_bootstrap": (i, [W, i, d, P(d), P(d), P(i), P(i)]),
            "or_epi_refine": (C.c_int64, [W, P(d), d, P(d), P(d)]),
            "or_ground_scale": (i, [W, d, d, P(d), P(d), P(C.c_int64)]),
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
                   hyps_per_frame=S, groups_per_frame=4 * S if G is None else G,
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

    def epipolar_bootstrap(self, n_samples, baseline=1.0):
        """(status, T1, per-sample scores, chosen sample, chosen candidate)."""
        T1 = np.zeros(16)
        scores = np.zeros(n_samples)
        m, c = C.c_int(-1), C.c_int(-1)
        st = lib().or_epipolar_bootstrap(self.ref, n_samples, float(baseline), _dp(T1), _dp(scores),
                                         C.byref(m), C.byref(c))
        return st, T1.reshape(4, 4), scores, m.value, c.value

    def epi_sample(self, m):
        E = np.zeros(9)
        j = np.zeros(8, dtype=np.int64)
        ok = lib().or_epi_sample(self.ref, m, _dp(E), ptr(j, C.c_int64))
        return ok, E.reshape(3, 3), j

    def epi_score(self, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        return lib().or_epi_score(self.ref, _dp(E))

    def epi_refine(self, E, median):
        """(inlier count, refined E, inlier threshold)."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        out, thr = np.zeros(9), C.c_double(0.0)
        n = lib().or_epi_refine(self.ref, _dp(E), float(median), _dp(out), C.byref(thr))
        return n, out.reshape(3, 3), thr.value

    def ground_scale(self, camera_height, max_tilt_deg=10.0):
        """(status, scale, mode of log2 height, candidate pixels)."""
        s, m, n = C.c_double(0), C.c_double(0), C.c_int64(0)
        st = lib().or_ground_scale(self.ref, float(camera_height), float(np.deg2rad(max_tilt_deg)), C.byref(s),
                                   C.byref(m), C.byref(n))
        return st, s.value, m.value, n.value

    def epi_cheirality(self, R, t):
        R = np.ascontiguousarray(R, dtype=np.float64)
        t = np.ascontiguousarray(t, dtype=np.float64)
        return lib().or_epi_cheirality(self.ref, _dp(R), _dp(t))

    def frame_crit(self, t, j, depth):
        return lib().or_frame_crit(self.ref, t, j, depth)

    def frame_eval(self, t, j, depth):
        out = np.zeros(12)
        v = lib().or_frame_eval(self.ref, t, j, depth, _dp(out))
        return v, out

    def valid_pixels(self, t):
        """Pixels with a 3D-2D correspondence at frame t, in pixel order."""
        out = np.zeros(self.H * self.W, dtype=np.int64)
        n = lib().or_valid_pixels(self.ref, t, ptr(out, C.c_int64))
        return out[:n]

    def draw_group(self, k, t, g, valid):
        """(distinct, the group's three pixels) drawn from the list `valid`."""
        valid = np.ascontiguousarray(valid, dtype=np.int64)
        j = np.zeros(3, dtype=np.int64)
        ok = lib().or_draw_group(self.ref, k, t, g, ptr(valid, C.c_int64), valid.size, ptr(j, C.c_int64))
        return bool(ok), j

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


def essential_8pt(m0, m1):
    m0 = np.ascontiguousarray(m0, dtype=np.float64)
    m1 = np.ascontiguousarray(m1, dtype=np.float64)
    E = np.zeros(9)
    ok = lib().or_essential_8pt(_dp(m0), _dp(m1), _dp(E))
    return ok, E.reshape(3, 3)


def essential_project(E):
    E = np.ascontiguousarray(E, dtype=np.float64)
    out, U, V = np.zeros(9), np.zeros(9), np.zeros(9)
    ok = lib().or_essential_project(_dp(E), _dp(out), _dp(U), _dp(V))
    return ok, out.reshape(3, 3), U.reshape(3, 3), V.reshape(3, 3)


def sampson(E, m0, m1):
    E = np.ascontiguousarray(E, dtype=np.float64)
    return lib().or_sampson(_dp(E), _dp(np.ascontiguousarray(m0, dtype=np.float64)),
                            _dp(np.ascontiguousarray(m1, dtype=np.float64)))


def essential_candidates(U, V):
    R, t = np.zeros(36), np.zeros(12)
    lib().or_essential_candidates(_dp(np.ascontiguousarray(U, dtype=np.float64)),
                                  _dp(np.ascontiguousarray(V, dtype=np.float64)), _dp(R), _dp(t))
    return R.reshape(4, 3, 3), t.reshape(4, 3)


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64_10(ptr(c, C.c_uint64), ptr(k, C.c_uint64), ptr(out, C.c_uint64))
    return out


def fisk_logpdf(x, log_alpha, beta):
    return lib().or_fisk_logpdf(float(x), float(log_alpha), float(beta))


def gauss_logpdf(x, log_alpha):
    """Log density of the squared EPE under the Gaussian residual model with
    the Fisk median alpha = exp(log_alpha)."""
    return lib().or_gauss_logpdf(float(x), float(log_alpha))


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
