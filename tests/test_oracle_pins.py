"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against an independent source: scipy's Fisk and
matrix exponential, numpy's Philox4x64-10, a sympy resultant, brute-force
enumeration, or a noiseless synthetic scene whose answer is known exactly.
"""
import itertools
import math

import ctypes

import numpy as np
import pytest

from tests.conftest import fronto_parallel_window


# ---------------------------------------------------------------------------
# Philox4x64-10 (Salmon et al., SC'11) against numpy's implementation
# ---------------------------------------------------------------------------
def _inc(ctr):
    c = [int(x) for x in ctr]
    for i in range(4):
        c[i] = (c[i] + 1) % (1 << 64)
        if c[i] != 0:
            break
    return c


@pytest.mark.parametrize("ctr", [[0, 0, 0, 0], [1, 2, 3, 4], [(1 << 64) - 1, 5, 7, 9],
                                 [123456789, 0, 3, 1]])
def test_philox_matches_numpy(oracle_lib, ctr):
    key = np.array([0x0123456789ABCDEF, 0xFEDCBA9876543210], dtype=np.uint64)
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=key)
    raw = bg.random_raw(8)
    # numpy advances the counter before each block of four outputs
    c1 = _inc(ctr)
    c2 = _inc(c1)
    got = np.concatenate([oracle_lib.philox4x64_10(c1, key), oracle_lib.philox4x64_10(c2, key)])
    assert np.array_equal(got, raw)


# ---------------------------------------------------------------------------
# Fisk model (Eqs. 3-7)
# ---------------------------------------------------------------------------
def test_fisk_logpdf_matches_scipy(oracle_lib):
    from scipy import stats
    rng = np.random.default_rng(0)
    for _ in range(200):
        alpha = 10 ** rng.uniform(-3, 3)
        beta = rng.uniform(0.05, 1.0)
        x = alpha * 10 ** rng.uniform(-4, 4)
        ref = stats.fisk(c=beta, scale=alpha).logpdf(x)
        got = oracle_lib.fisk_logpdf(x, math.log(alpha), beta)
        assert got == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_fisk_normalised_and_median(oracle_lib):
    from scipy import integrate
    for alpha, beta in [(0.01, 1.0), (0.0246, 0.978), (0.37, 0.912), (3.0, 0.5)]:
        f = lambda x: math.exp(oracle_lib.fisk_logpdf(x, math.log(alpha), beta))
        # substitute x = alpha e^s so that the heavy tail is integrable by quad
        g = lambda s: f(alpha * math.exp(s)) * alpha * math.exp(s)
        total, _ = integrate.quad(g, -200, 200, limit=400)
        below, _ = integrate.quad(g, -200, 0, limit=400)
        assert total == pytest.approx(1.0, abs=1e-8)
        assert below == pytest.approx(0.5, abs=1e-8)      # the median is alpha


def test_lambda_is_the_indistinguishable_epe(oracle_lib):
    """Sec. 4: lambda is the EPE fraction at which W = 0.5, i.e. rho = mu when
    |xi - v_ob| = lambda |v_ob|. Flows are set to xi / (1 + lambda)."""
    flows, K, poses, depth = fronto_parallel_window(T=2)
    lam = 0.15
    xi = flows.copy()
    flows = xi / (1.0 + lam)
    ow = oracle_lib.OracleWindow(flows, K, S=8)
    ow.theta[:] = depth
    ow.poses[:] = poses
    H, W = depth.shape
    for t in (1, 2):
        for j in [0, 5, W + 3, H * W // 2]:
            v, o = ow.frame_eval(t, j, depth.flat[j])
            if v < 2:
                continue
            assert o[6] == pytest.approx(o[7], rel=1e-12)        # log rho == log mu
            assert o[8] == pytest.approx(math.log(0.5), abs=1e-12)


def test_mie_term_at_long_flows_matches_scipy(oracle_lib):
    """Past |v_ob| = 454.5 px the shape B = b1 |v_ob| + b2 of Eq. 6 would be
    non-positive; the oracle floors it at beta_min (reading 3) while the scale
    alpha = a1 e^{a2 |v_ob|} of Eq. 5 keeps growing. At flows of 500-6000 px
    the per-(t, j) MIE term log rho/(rho + mu) must equal the one scipy's Fisk
    density gives with that beta and alpha, the residual and lambda^2 |v|^2
    (Eq. 7) clamped as the oracle clamps them."""
    from scipy import stats
    from tests.helpers import small_window
    w = small_window(seed=1000, W=64, H=48, f=48.0, T=2)
    rng = np.random.default_rng(5)
    fl = w.flows.astype(np.float64).copy()
    mag = rng.uniform(500.0, 6000.0, size=fl.shape[:3])
    ang = rng.uniform(0.0, 2.0 * np.pi, size=fl.shape[:3])
    fl[..., 0], fl[..., 1] = mag * np.cos(ang), mag * np.sin(ang)
    ow = oracle_lib.OracleWindow(fl, w.K)
    ow.poses[:] = w.poses
    p = oracle_lib.PAPER_DEFAULTS
    checked = 0
    for _ in range(200):
        t = int(rng.integers(1, w.T + 1))
        j = int(rng.integers(0, w.W * w.H))
        depth = float(w.depth0.flat[j] * rng.uniform(0.8, 1.2))
        v, diag = ow.frame_eval(t, j, depth)
        if v < 2:
            continue
        res, vob = diag[0:2], diag[4:6]
        n = np.hypot(*vob)                 # bilinear between long flows: mostly, not always, > 454.5
        beta = max(p["b1"] * n + p["b2"], p["beta_min"])
        alpha = p["a1"] * np.exp(p["a2"] * n)
        x = np.clip(res @ res, p["x_min"], p["x_max"])
        x_mu = np.clip(p["lambda_"] ** 2 * n * n, p["x_min"], p["x_max"])
        ref = -np.logaddexp(0.0, stats.fisk.logpdf(x_mu, beta, scale=alpha) - stats.fisk.logpdf(x, beta, scale=alpha))
        assert ow.frame_crit(t, j, depth) == pytest.approx(ref, rel=1e-9, abs=1e-12)
        checked += n > 454.5
    assert checked > 20


# ---------------------------------------------------------------------------
# Geometry, bilinear sampling, triangulation
# ---------------------------------------------------------------------------
def test_bilinear_reproduces_affine_fields(oracle_lib):
    H, W, T = 9, 11, 2
    ys, xs = np.mgrid[0:H, 0:W].astype(float)
    flows = np.zeros((T, H, W, 2))
    flows[0, ..., 0] = 0.3 + 0.02 * xs - 0.05 * ys
    flows[0, ..., 1] = -1.1 + 0.07 * xs + 0.01 * ys
    ow = oracle_lib.OracleWindow(flows, (10.0, 10.0, 5.0, 4.0), S=4)
    import ctypes
    rng = np.random.default_rng(1)
    for _ in range(100):
        u, v = rng.uniform(0, W - 1), rng.uniform(0, H - 1)
        out = np.zeros(2)
        ok = oracle_lib.lib().or_bilinear(ow.ref, 1, u, v, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert ok == 1
        assert out[0] == pytest.approx(0.3 + 0.02 * u - 0.05 * v, abs=1e-13)
        assert out[1] == pytest.approx(-1.1 + 0.07 * u + 0.01 * v, abs=1e-13)
    out = np.zeros(2)
    p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert oracle_lib.lib().or_bilinear(ow.ref, 1, W - 1.0, H - 1.0, p) == 1
    assert oracle_lib.lib().or_bilinear(ow.ref, 1, W - 1.0 + 1e-9, 0.0, p) == 0
    assert oracle_lib.lib().or_bilinear(ow.ref, 1, -1e-9, 0.0, p) == 0


def test_noiseless_residual_is_zero(oracle_lib):
    flows, K, poses, depth = fronto_parallel_window(T=3)
    ow = oracle_lib.OracleWindow(flows, K, S=8)
    ow.theta[:] = depth
    ow.poses[:] = poses
    H, W = depth.shape
    n_valid = 0
    for t in (1, 2, 3):
        for j in range(H * W):
            v, o = ow.frame_eval(t, j, depth.flat[j])
            if v == 2:
                n_valid += 1
                assert abs(o[0]) < 1e-9 and abs(o[1]) < 1e-9
    assert n_valid > 0.8 * 3 * H * W


def test_noiseless_residual_first_frame_general_scene(oracle_lib):
    from paper_2104_06789_gb300 import synthetic as sy
    w = sy.small_planes(noise=False, nonrigid=False)
    ow = oracle_lib.OracleWindow(w.flows, w.K, S=8)
    ow.theta[:] = w.depth0
    ow.poses[:] = w.poses
    for j in range(0, w.H * w.W, 13):
        v, o = ow.frame_eval(1, j, w.depth0.flat[j])
        if v == 2:
            assert abs(o[0]) < 1e-9 and abs(o[1]) < 1e-9


def test_triangulation_noiseless(oracle_lib):
    from paper_2104_06789_gb300 import synthetic as sy
    w = sy.small_planes(noise=False, nonrigid=False)
    ow = oracle_lib.OracleWindow(w.flows, w.K, S=8, inv_depth_min=1e-3, inv_depth_max=10.0)
    ow.bootstrap(w.poses[0])
    rel = np.abs(ow.theta - w.depth0) / w.depth0
    assert np.max(rel) < 1e-10
    assert np.all(ow.wmap == 1.0)
    assert np.allclose(ow.poses, w.poses[0])


def test_triangulation_without_parallax_goes_far(oracle_lib):
    flows, K, poses, depth = fronto_parallel_window(T=1)
    ow = oracle_lib.OracleWindow(np.zeros_like(flows), K, S=8, inv_depth_min=0.05, inv_depth_max=2.0)
    ow.bootstrap(poses[0])
    assert np.allclose(ow.theta, 1 / 0.05)
    # negative depth (flow opposite to the translation) also goes far
    ow = oracle_lib.OracleWindow(-flows, K, S=8, inv_depth_min=0.05, inv_depth_max=2.0)
    ow.bootstrap(poses[0])
    assert np.allclose(ow.theta, 1 / 0.05)


def test_triangulation_clamps_to_the_depth_range(oracle_lib):
    """Reading 19: the bootstrap's inverse depth is clamped to [inv_min,
    inv_max]. On a noiseless window, whose triangulation is exact (the pin
    above), a range set inside the scene's puts the nearest pixels exactly on
    1/inv_max, the farthest on 1/inv_min, and leaves every other depth exact."""
    from paper_2104_06789_gb300 import synthetic as sy
    w = sy.small_planes(noise=False, nonrigid=False)
    inv = 1.0 / w.depth0
    lo, hi = 0.07, 0.3                        # the scene spans inverse depths 0.05 (background) to 0.48
    ow = oracle_lib.OracleWindow(w.flows, w.K, S=8, inv_depth_min=lo, inv_depth_max=hi)
    ow.bootstrap(w.poses[0])
    expect = 1.0 / np.clip(inv, lo, hi)
    assert np.max(np.abs(ow.theta - expect) / expect) < 1e-10
    assert np.any(inv > hi) and np.any(inv < lo)


# ---------------------------------------------------------------------------
# P3P (Eq. 17)
# ---------------------------------------------------------------------------
def _random_rotation(rng, max_angle):
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    a = rng.uniform(0, max_angle)
    Kx = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(a) * Kx + (1 - math.cos(a)) * Kx @ Kx


def _p3p_instance(rng):
    R = _random_rotation(rng, 0.5)
    t = rng.normal(size=3) * 0.5
    while True:
        P = np.column_stack([rng.uniform(-3, 3, 3), rng.uniform(-3, 3, 3), rng.uniform(4, 12, 3)])
        Q = P @ R.T + t
        if np.all(Q[:, 2] > 0.5):
            break
    b = Q / np.linalg.norm(Q, axis=1, keepdims=True)
    return R, t, P, b


def test_p3p_recovers_generating_pose(oracle_lib):
    rng = np.random.default_rng(7)
    for _ in range(300):
        R, t, P, b = _p3p_instance(rng)
        Rs, ts, s1 = oracle_lib.p3p(P, b)
        assert len(Rs) >= 1
        err = [max(np.abs(Ri - R).max(), np.abs(ti - t).max()) for Ri, ti in zip(Rs, ts)]
        assert min(err) < 1e-9
        assert np.all(np.diff(s1) >= 0)
        for Ri, ti in zip(Rs, ts):
            Qi = P @ Ri.T + ti
            assert np.all(Qi[:, 2] > 0)
            bi = Qi / np.linalg.norm(Qi, axis=1, keepdims=True)
            assert np.abs(bi - b).max() < 1e-8
            assert np.abs(Ri @ Ri.T - np.eye(3)).max() < 1e-9


def _sympy_p3p_s1(P, b):
    """All positive solutions (s1, s2, s3) of the three law-of-cosines
    equations, by sympy resultants in exact rational arithmetic."""
    import sympy as sp
    s1, s2, s3 = sp.symbols("s1 s2 s3")
    Rq = lambda x: sp.Rational(float(x))
    d = lambda i, j: Rq(np.sum((P[i] - P[j]) ** 2))
    c = lambda i, j: Rq(np.dot(b[i], b[j]))
    e12 = s1**2 + s2**2 - 2 * c(0, 1) * s1 * s2 - d(0, 1)
    e13 = s1**2 + s3**2 - 2 * c(0, 2) * s1 * s3 - d(0, 2)
    e23 = s2**2 + s3**2 - 2 * c(1, 2) * s2 * s3 - d(1, 2)
    r = sp.resultant(sp.resultant(e12, e23, s2), e13, s3)
    poly = sp.Poly(r, s1)
    out = []
    for root in poly.nroots(n=30, maxsteps=200):
        if abs(sp.im(root)) > 1e-12 or sp.re(root) <= 0:
            continue
        v1 = float(sp.re(root))
        # back-substitute: s2 from e12, s3 from e13, keep the consistent positive pair
        c12, c13, c23 = float(c(0, 1)), float(c(0, 2)), float(c(1, 2))
        d12, d13, d23 = float(d(0, 1)), float(d(0, 2)), float(d(1, 2))
        for sgn2, sgn3 in itertools.product((-1, 1), repeat=2):
            disc2 = (c12 * v1) ** 2 - (v1**2 - d12)
            disc3 = (c13 * v1) ** 2 - (v1**2 - d13)
            if disc2 < 0 or disc3 < 0:
                continue
            v2 = c12 * v1 + sgn2 * math.sqrt(disc2)
            v3 = c13 * v1 + sgn3 * math.sqrt(disc3)
            if v2 <= 0 or v3 <= 0:
                continue
            if abs(v2**2 + v3**2 - 2 * c23 * v2 * v3 - d23) < 1e-6 * max(1.0, d23):
                out.append(v1)
    return sorted(set(round(x, 9) for x in out))


def test_p3p_solution_set_matches_sympy_resultant(oracle_lib):
    rng = np.random.default_rng(11)
    for _ in range(6):
        R, t, P, b = _p3p_instance(rng)
        _, _, s1 = oracle_lib.p3p(P, b)
        ref = _sympy_p3p_s1(P, b)
        assert [round(x, 9) for x in s1] == pytest.approx(ref, abs=2e-9)


# ---------------------------------------------------------------------------
# se(3)
# ---------------------------------------------------------------------------
def test_se3_exp_matches_matrix_exponential(oracle_lib):
    from scipy.linalg import expm
    rng = np.random.default_rng(3)
    for scale in (1e-9, 1e-5, 0.3, 2.5):
        for _ in range(10):
            p = rng.normal(size=6) * scale
            rho, phi = p[:3], p[3:]
            M = np.zeros((4, 4))
            M[:3, :3] = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
            M[:3, 3] = rho
            E = expm(M)
            R, t = oracle_lib.se3_exp(p)
            assert np.abs(R - E[:3, :3]).max() < 1e-12
            assert np.abs(t - E[:3, 3]).max() < 1e-12 * max(1.0, np.abs(t).max())


def test_se3_log_round_trip(oracle_lib):
    rng = np.random.default_rng(4)
    cases = [rng.normal(size=6) * s for s in (1e-9, 1e-5, 0.1, 1.0) for _ in range(5)]
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    cases.append(np.concatenate([[0.3, -0.2, 0.1], ax * (math.pi - 1e-6)]))
    cases.append(np.concatenate([[0.3, -0.2, 0.1], ax * (math.pi - 1e-2)]))
    for p in cases:
        if np.linalg.norm(p[3:]) >= math.pi:
            continue
        R, t = oracle_lib.se3_exp(p)
        q = oracle_lib.se3_log(R, t)
        tol = 1e-12 if np.linalg.norm(p[3:]) < math.pi - 1e-3 else 1e-7
        assert np.abs(q - p).max() < tol * max(1.0, np.abs(p).max())


# ---------------------------------------------------------------------------
# Meanshift (Eqs. 18-19)
# ---------------------------------------------------------------------------
def test_meanshift_single_and_symmetric(oracle_lib):
    p = np.array([[0.1, 0.2, 0.3, 0.01, 0.02, 0.03]])
    it, x = oracle_lib.meanshift(p, np.ones(1), 0, 0.1, 0.004)
    assert np.array_equal(x, p[0])
    p = np.array([[0.0] * 6, [0.05, 0, 0, 0.01, 0, 0]])
    it, x = oracle_lib.meanshift(p, np.ones(2), 0, 0.1, 0.004, max_iter=10000, tol=1e-15)
    assert np.abs(x - p.mean(0)).max() < 1e-12


def test_meanshift_converges_to_stationary_point(oracle_lib):
    rng = np.random.default_rng(5)
    st, sr = 0.1, 0.004
    p = np.concatenate([rng.normal(size=(40, 6)) * 0.2, rng.normal(size=(40, 6)) * 0.05 + 1.0])
    p[:, 3:] *= 0.1
    w = rng.uniform(0.1, 1.0, size=len(p))
    it, x = oracle_lib.meanshift(p, w, 0, st, sr, max_iter=100000, tol=1e-14)
    inv = np.array([1 / st] * 3 + [1 / sr] * 3)

    def kde(y):
        d = y - p
        return np.sum(w * np.exp(-0.5 * np.sum(d * d * inv, axis=1)))

    h = 1e-6
    for i in range(6):
        e = np.zeros(6)
        e[i] = h * (np.sqrt(st) if i < 3 else np.sqrt(sr))
        g = (kde(x + e) - kde(x - e)) / (2 * e[i])
        assert abs(g) < 1e-6 * kde(x) / np.sqrt(1 / inv[i])


# ---------------------------------------------------------------------------
# Forward-backward (Eqs. 11-14)
# ---------------------------------------------------------------------------
def _brute_marginals(w, gamma):
    L = len(w)
    num = np.zeros(L)
    Z = 0.0
    for lab in itertools.product((0, 1), repeat=L):
        p = 0.5
        for j, l in enumerate(lab):
            p *= w[j] if l else (1 - w[j])
            if j:
                p *= gamma if l == lab[j - 1] else 1 - gamma
        Z += p
        num += p * np.array(lab)
    return num / Z


@pytest.mark.parametrize("L", [1, 2, 5, 10])
def test_forward_backward_brute_force(oracle_lib, L):
    rng = np.random.default_rng(L)
    for gamma in (0.9, 0.6, 0.99):
        w = rng.uniform(0.01, 0.99, size=L)
        q = oracle_lib.forward_backward(w, gamma)
        assert np.abs(q - _brute_marginals(w, gamma)).max() < 1e-12


@pytest.mark.parametrize("axis", [0, 1])
def test_smoothing_runs_independent_chains_along_rows_or_columns(oracle_lib, axis):
    """The E-step smooths each frame's emissions on 1-D chains (Eqs. 11-14):
    along image rows for axis 0 (horizontal sweeps) and columns for axis 1,
    frames independent (readings 8, 10). Every chain of a 5 x 4 window with
    T = 2 against brute-force enumeration of its 2^L labelings."""
    from paper_2104_06789_gb300 import synthetic as sy
    w = sy.small_planes(W=5, H=4, f=4.0, T=2, seed=1006)
    ow = oracle_lib.OracleWindow(w.flows, w.K, S=8)
    rng = np.random.default_rng(17 + axis)
    emis = rng.uniform(0.01, 0.99, size=(w.T, w.H, w.W))
    q = ow.smooth(axis, emis)
    g = oracle_lib.PAPER_DEFAULTS["gamma"]
    for t in range(w.T):
        chains = emis[t] if axis == 0 else emis[t].T
        out = q[t] if axis == 0 else q[t].T
        for c in range(chains.shape[0]):
            assert np.abs(out[c] - _brute_marginals(chains[c], g)).max() < 1e-12


def test_forward_backward_special_cases(oracle_lib):
    rng = np.random.default_rng(9)
    w = rng.uniform(0.01, 0.99, size=50)
    assert np.abs(oracle_lib.forward_backward(w, 0.5) - w).max() < 1e-14
    q = oracle_lib.forward_backward(w, 1.0 - 1e-12)
    assert np.ptp(q) < 1e-9


# ---------------------------------------------------------------------------
# Random draws
# ---------------------------------------------------------------------------
def test_depth_samples_uniform_in_inverse_depth(oracle_lib):
    from scipy import stats
    flows, K, poses, depth = fronto_parallel_window(W=100, H=100, T=1)
    ow = oracle_lib.OracleWindow(flows, K, S=8, inv_depth_min=0.1, inv_depth_max=2.0)
    inv = np.array([1.0 / ow.depth_sample(3, j) for j in range(10000)])
    assert inv.min() >= 0.1 and inv.max() < 2.0
    assert stats.kstest((inv - 0.1) / 1.9, "uniform").pvalue > 1e-3


def test_group_draws_uniform(oracle_lib):
    """Group pixels are uniform over the list handed to the draw and distinct
    with the birthday probability of three draws from n."""
    from scipy import stats
    flows, K, poses, depth = fronto_parallel_window(W=10, H=10, T=1)
    ow = oracle_lib.OracleWindow(flows, K, S=8)
    valid = np.arange(3, 100, 2, dtype=np.int64)          # any increasing list
    n = valid.size
    counts = np.zeros(100)
    distinct = 0
    for g in range(5000):
        ok, j = ow.draw_group(2, 1, g, valid)
        distinct += ok
        counts[j] += 1
    assert counts[np.setdiff1d(np.arange(100), valid)].sum() == 0
    assert stats.chisquare(counts[valid]).pvalue > 1e-3
    assert distinct == pytest.approx(5000 * (1 - 1 / n) * (1 - 2 / n), rel=0.02)
    ok, _ = ow.draw_group(2, 1, 0, np.zeros(0, dtype=np.int64))
    assert not ok


def test_valid_pixels_are_the_correspondences(oracle_lib):
    """V_t lists, in pixel order, exactly the pixels whose pi_{t-1} lies inside
    I_{t-1} in front of camera t-1 (checked per pixel through or_frame_ell's
    validity report); from frame 2 on the pixels that the earlier motion
    carries out of the image drop out of the list."""
    flows, K, poses, depth = fronto_parallel_window(W=24, H=18, T=3)
    ow = oracle_lib.OracleWindow(flows, K, S=8)
    ow.theta[:] = depth
    ow.poses[:] = poses
    for t in (1, 2, 3):
        v = ow.valid_pixels(t)
        assert np.all(np.diff(v) > 0)
        brute = []
        for j in range(depth.size):
            flag = ctypes.c_int(0)
            oracle_lib.lib().or_frame_ell(ow.ref, t, j, float(ow.theta.flat[j]), ctypes.byref(flag))
            if flag.value >= 1:
                brute.append(j)
        assert np.array_equal(v, np.array(brute, dtype=np.int64))
    assert ow.valid_pixels(1).size == depth.size            # pi_0 is the pixel itself
    assert 0 < ow.valid_pixels(2).size < depth.size


def test_every_frame_collects_exactly_S(oracle_lib):
    """With the draws over V_t, every frame of a driving-like window collects
    exactly S hypotheses within the 4 S group budget, from groups whose three
    pixels all have a correspondence, in increasing group order."""
    from paper_2104_06789_gb300 import synthetic as sy
    w = sy.driving(W=207, H=63, f=119.7, T=8, seed=3000)
    S = 512
    ow = oracle_lib.OracleWindow(w.flows, w.K, S=S, inv_depth_min=w.inv_depth_range[0],
                                 inv_depth_max=w.inv_depth_range[1])
    ow.bootstrap(w.poses[0])
    ow.poses[:] = w.poses
    for t in range(1, w.T + 1):
        valid = set(ow.valid_pixels(t).tolist())
        assert len(valid) < w.W * w.H or t == 1
        R, tv, wt, grp, slot = ow.collect_hypotheses(0, t)
        assert len(grp) == S, (t, len(grp))
        assert np.all(np.diff(grp) >= 0) and grp[-1] < 4 * S
        for g in np.unique(grp)[:20]:
            ok, j = ow.draw_group(0, t, int(g), ow.valid_pixels(t))
            assert ok and all(int(x) in valid for x in j)


# ---------------------------------------------------------------------------
# Dense scoring, MIE sweep, full loop
# ---------------------------------------------------------------------------
def test_dense_score_peaks_at_true_pose(oracle_lib):
    from paper_2104_06789_gb300 import synthetic as sy
    w = sy.small_planes(noise=False, nonrigid=False, W=40, H=30, f=30.0)
    ow = oracle_lib.OracleWindow(w.flows, w.K, S=8)
    ow.theta[:] = w.depth0
    ow.poses[:] = w.poses
    t = 2
    R0, t0 = w.poses[t - 1][:3, :3], w.poses[t - 1][:3, 3]
    rng = np.random.default_rng(2)
    Rs, ts = [R0], [t0]
    for _ in range(6):
        Rs.append(_random_rotation(rng, 0.01) @ R0)
        ts.append(t0 + rng.normal(size=3) * 0.01)
    L = ow.score(t, np.array(Rs), np.array(ts))
    assert np.argmax(L) == 0
    assert np.all(L <= 0)
    # doubling the rigidness weights doubles every score (L is linear in W)
    ow.wmap[:] = 0.5
    L2 = ow.score(t, np.array(Rs), np.array(ts))
    assert np.allclose(L2 * 2, L, rtol=1e-14)


def test_dense_score_is_the_weighted_sum_of_the_pinned_terms(oracle_lib):
    """L_h (the Eq. 10 criterion with the pose as the free variable) sums, over
    the pixels whose pi_{t-1} is valid, the unsmoothed W_t^j times the
    per-(t, j) term that the Fisk pins check against scipy, evaluated at T_t = h;
    pixels without a correspondence add nothing and a point behind camera t
    adds log 1/2. Checked on a noisy window with random W against the per-term
    function (frame_crit) with the hypothesis set as the frame's pose."""
    from paper_2104_06789_gb300 import synthetic as sy
    w = sy.small_planes(W=24, H=18, f=18.0, T=3, seed=1003)
    ow = oracle_lib.OracleWindow(w.flows, w.K, S=8)
    rng = np.random.default_rng(9)
    ow.theta[:] = w.depth0 * rng.uniform(0.8, 1.2, size=w.depth0.shape)
    ow.wmap[:] = rng.uniform(0.0, 1.0, size=ow.wmap.shape)
    ow.poses[:] = w.poses
    t = 3
    R0, t0 = w.poses[t - 1][:3, :3], w.poses[t - 1][:3, 3]
    hyps = [(R0, t0), (_random_rotation(rng, 0.05) @ R0, t0 + rng.normal(size=3) * 0.05),
            (R0, t0 + np.array([0.0, 0.0, -30.0]))]             # the last puts points behind camera t
    L = ow.score(t, np.array([h[0] for h in hyps]), np.array([h[1] for h in hyps]))
    behind = 0
    for (R, tv), Lh in zip(hyps, L):
        ow.poses[t - 1][:3, :3], ow.poses[t - 1][:3, 3] = R, tv
        ref = 0.0
        for j in range(w.W * w.H):
            v, _ = ow.frame_eval(t, j, float(ow.theta.flat[j]))
            if v >= 1:                                            # pi_{t-1} valid
                c = ow.frame_crit(t, j, float(ow.theta.flat[j]))
                behind += v == 1 and c == pytest.approx(math.log(0.5))
                ref += ow.wmap[t - 1].flat[j] * c
        assert Lh == pytest.approx(ref, rel=1e-12)
    assert behind > 0


def test_rigidness_update_is_the_per_pixel_posterior(oracle_lib):
    """The unsmoothed rigidness update (Table 1, last line; reading 11) sets
    every W_t^j to the posterior rho/(rho + mu) of the rigid hypothesis under
    a uniform prior, at the current depth and poses: rho the Fisk density of
    the squared residual, mu that of lambda^2 |v_ob|^2 (Eqs. 3-7), from scipy;
    1/2 where the pixel has no observation at pi_{t-1} or lies behind camera
    t. Every (t, j) of a noisy window with a perturbed depth."""
    from scipy import stats
    from paper_2104_06789_gb300 import synthetic as sy
    w = sy.small_planes(W=24, H=18, f=18.0, T=3, seed=1004)
    ow = oracle_lib.OracleWindow(w.flows, w.K, S=8)
    rng = np.random.default_rng(11)
    ow.theta[:] = w.depth0 * rng.uniform(0.9, 1.1, size=w.depth0.shape)
    ow.poses[:] = w.poses
    ow.wmap[:] = rng.uniform(0.0, 1.0, size=ow.wmap.shape)      # overwritten by the update
    expect = np.zeros_like(ow.wmap)
    p = oracle_lib.PAPER_DEFAULTS
    n_none = 0
    for t in range(1, w.T + 1):
        for j in range(w.W * w.H):
            v, diag = ow.frame_eval(t, j, float(ow.theta.flat[j]))
            if v < 2:
                expect[t - 1].flat[j] = 0.5
                n_none += 1
                continue
            res, vob = diag[0:2], diag[4:6]
            n = np.hypot(*vob)
            alpha = p["a1"] * np.exp(p["a2"] * n)
            beta = max(p["b1"] * n + p["b2"], p["beta_min"])
            x = np.clip(res @ res, p["x_min"], p["x_max"])
            x_mu = np.clip(p["lambda_"] ** 2 * n * n, p["x_min"], p["x_max"])
            lr = stats.fisk.logpdf(x, beta, scale=alpha)
            lm = stats.fisk.logpdf(x_mu, beta, scale=alpha)
            expect[t - 1].flat[j] = 1.0 / (1.0 + np.exp(lm - lr))
    ow.rigidness()
    assert np.allclose(ow.wmap, expect, rtol=1e-10, atol=1e-14)
    assert 0 < n_none < expect.size                             # both conventions occur


def test_sweep_candidate_score_is_the_q_weighted_sum_over_frames(oracle_lib):
    """The depth sweep scores a candidate depth d of pixel j by Eq. 10,
    sum over t of q_t^j times the per-(t, j) term at d (the scipy-pinned
    term; log 1/2 where the pixel has no observation or lies behind camera t),
    with q the smoothed rigidness. Random q, depths around the truth and far
    off, every pixel of a small noisy window."""
    from paper_2104_06789_gb300 import synthetic as sy
    w = sy.small_planes(W=20, H=15, f=15.0, T=3, seed=1005)
    ow = oracle_lib.OracleWindow(w.flows, w.K, S=8)
    ow.poses[:] = w.poses
    rng = np.random.default_rng(13)
    q = rng.uniform(0.0, 1.0, size=(w.T, w.H, w.W))
    for j in range(w.W * w.H):
        for d in (float(w.depth0.flat[j]) * rng.uniform(0.7, 1.3), float(rng.uniform(0.5, 50.0))):
            ref = sum(q[t - 1].flat[j] * ow.frame_crit(t, j, d) for t in range(1, w.T + 1))
            assert ow.mie_score(q, j, d) == pytest.approx(ref, rel=1e-12, abs=1e-15)


def test_mie_sweep_monotone_and_fixed_point(oracle_lib):
    flows, K, poses, depth = fronto_parallel_window(T=3)
    ow = oracle_lib.OracleWindow(flows, K, S=8, inv_depth_min=0.05, inv_depth_max=1.0)
    ow.theta[:] = depth
    ow.poses[:] = poses
    q = np.ones((3,) + depth.shape)
    labels = ow.mie_sweep(0, q)
    assert np.all(labels == 0)
    assert np.array_equal(ow.theta, depth)
    # perturbed start: the chosen score never falls below the previous depth's
    rng = np.random.default_rng(0)
    start = depth * rng.uniform(0.7, 1.4, size=depth.shape)
    for k in range(4):
        ow.theta[:] = start
        before = np.array([ow.mie_score(q, j, start.flat[j]) for j in range(depth.size)])
        ow.mie_sweep(k, q)
        after = np.array([ow.mie_score(q, j, ow.theta.flat[j]) for j in range(depth.size)])
        assert np.all(after >= before)


def test_full_loop_noiseless_fixed_point(oracle_lib):
    """A noiseless scene with an exact bootstrap is a fixed point: with a
    kernel narrow enough that spurious P3P roots carry no mass, the poses stay
    at the truth and the depth does not move."""
    flows, K, poses, depth = fronto_parallel_window(W=24, H=18, T=3)
    ow = oracle_lib.OracleWindow(flows, K, S=32, inv_depth_min=0.05, inv_depth_max=1.0,
                                 sigma_t=1e-8, sigma_r=1e-10)
    ow.bootstrap(poses[0])
    assert np.max(np.abs(ow.theta - depth)) < 1e-12
    st = ow.run(0, 2)
    assert st == 0
    assert np.abs(ow.poses - poses).max() < 1e-9
    assert np.max(np.abs(ow.theta - depth)) < 1e-12


def test_full_loop_is_scale_equivariant(oracle_lib):
    """A monocular window fixes the scene only up to scale, and the loop takes
    its scale from T_1 (Sec. 5.3): on a noisy window, scaling T_1's
    translation, the depth-sample range and the translation variance of the
    pose kernel (a length squared, Eq. 18) by s = 2, 2 and 4 must scale every
    depth and translation of two full iterations by exactly 2 and leave the
    rotations and rigidness maps unchanged; only the meanshift's stopping test
    on the mixed (translation, rotation) step is not scale-free, so poses and
    rigidness agree to its tolerance. Unit-inconsistent arithmetic anywhere in
    the loop (a variance read as a standard deviation, the translation and
    rotation variances swapped: both checked by planting them) breaks it."""
    from tests.helpers import small_window
    w = small_window(seed=1000, W=48, H=36, f=36.0, T=3)
    flows = w.flows.astype(np.float64)

    def run(s):
        T1 = w.poses[0].copy()
        T1[:3, 3] *= s
        ow = oracle_lib.OracleWindow(flows, w.K, S=64, inv_depth_min=w.inv_depth_range[0] / s,
                                     inv_depth_max=w.inv_depth_range[1] / s, sigma_t=0.1 * s * s)
        ow.bootstrap(T1)
        assert ow.run(0, 2) == 0
        return ow

    a, b = run(1.0), run(2.0)
    assert np.array_equal(b.theta, 2.0 * a.theta)
    assert np.abs(b.poses[:, :3, 3] - 2.0 * a.poses[:, :3, 3]).max() < 1e-9
    assert np.abs(b.poses[:, :3, :3] - a.poses[:, :3, :3]).max() < 1e-9
    assert np.abs(b.wmap - a.wmap).max() < 1e-7


# ---------------------------------------------------------------------------
# MIE sweep: neighbour propagation (Fig. 5, Sec. 5.1)
# ---------------------------------------------------------------------------
def _chain_starts(W, H, k):
    """Pixel indices of the first position of every chain of direction k mod 4
    ([left to right, top to bottom, right to left, bottom to top])."""
    d = k % 4
    if d == 0:
        return [r * W for r in range(H)]
    if d == 1:
        return list(range(W))
    if d == 2:
        return [r * W + W - 1 for r in range(H)]
    return [(H - 1) * W + c for c in range(W)]


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_mie_sweep_propagates_the_chain_winner(oracle_lib, k):
    """Only each chain's first pixel starts at the true depth; every other
    pixel starts wrong, and the depth samples cannot reach the truth (inverse
    depth range [0.3, 1] excludes 1/5). One sweep must carry the truth down
    every chain through the neighbour candidate: each later pixel is labelled
    nbr and holds the true depth exactly, the chain starts keep theirs (prev).
    Taking the neighbour from the pre-sweep depth, running a chain backwards
    or dropping the candidate all leave wrong depths behind."""
    flows, K, poses, depth = fronto_parallel_window(W=24, H=18, T=3)
    H, W = depth.shape
    ow = oracle_lib.OracleWindow(flows, K, S=8, inv_depth_min=0.3, inv_depth_max=1.0)
    ow.poses[:] = poses
    ow.theta[:] = 2.0
    starts = _chain_starts(W, H, k)
    ow.theta.flat[starts] = 5.0
    q = np.ones((3, H, W))
    labels = ow.mie_sweep(k, q)
    expect = np.ones(H * W, dtype=np.uint8)
    expect[starts] = 0
    assert np.array_equal(labels.ravel(), expect)
    assert np.all(ow.theta == 5.0)


# ---------------------------------------------------------------------------
# Pose hypotheses: weights (Eq. 19) and the meanshift seed
# ---------------------------------------------------------------------------
def test_hypothesis_weight_is_the_product_of_the_groups_rigidness(oracle_lib):
    """Each hypothesis carries prod_i W_t(j_i) over the three pixels of its
    group, with the unsmoothed W of its own frame t (Eq. 19): W is set by hand
    to distinct values per (t, j), the group's pixels are re-drawn from the
    frame's valid list, and the product is compared exactly."""
    flows, K, poses, depth = fronto_parallel_window(W=24, H=18, T=3)
    ow = oracle_lib.OracleWindow(flows, K, S=96, inv_depth_min=0.05, inv_depth_max=1.0)
    ow.theta[:] = depth
    ow.poses[:] = poses
    rng = np.random.default_rng(19)
    ow.wmap[:] = rng.uniform(0.05, 1.0, size=ow.wmap.shape)
    for t in (1, 2, 3):
        valid = ow.valid_pixels(t)
        R, tv, wts, grp, slot = ow.collect_hypotheses(1, t)
        assert len(grp) == 96
        for h in range(len(grp)):
            ok, j = ow.draw_group(1, t, int(grp[h]), valid)
            Wt = ow.wmap[t - 1].ravel()
            assert ok and wts[h] == Wt[j[0]] * Wt[j[1]] * Wt[j[2]]
        assert len(np.unique(wts)) > 10


def _two_motion_window(W=40, H=30, f=30.0, depth=5.0, split=0.7, tA=(0.05, -0.03), tB=(-1.0, 0.8)):
    """A fronto-parallel plane whose left `split` of the columns moves with
    the camera translation tA and whose other columns move as if the camera
    had translated by tB (a second rigid motion): noiseless P3P groups inside
    either region return that region's pose exactly."""
    K = (f, f, (W - 1) / 2.0, (H - 1) / 2.0)
    flows = np.zeros((1, H, W, 2))
    cols = int(round(split * W))
    flows[0, :, :cols] = [f * tA[0] / depth, f * tA[1] / depth]
    flows[0, :, cols:] = [f * tB[0] / depth, f * tB[1] / depth]
    TA, TB = np.eye(4), np.eye(4)
    TA[:2, 3] = tA
    TB[:2, 3] = tB
    return flows, K, TA, TB, np.full((H, W), depth), cols


def test_meanshift_is_seeded_at_the_best_dense_score(oracle_lib):
    """Two rigid motions: region A (70 % of the pixels, W = 0.6) moves with the
    camera pose TA, region B (30 %, W = 1) with TB, their flows 7.7 px apart.
    By hand: under TA the residual is zero on A and 7.7 px on B; under TB the
    same residual falls on A. The weighted pixel count puts 0.3 N under the
    penalty for TA against 0.42 N for TB, and A's small observed flow
    (0.35 px: a small Fisk scale alpha, Eq. 5) makes each of TB's penalties
    the larger one, so the dense score's argmax lies in A's cluster. The
    heaviest hypotheses (Eq. 19: 1 in B, 0.216 in A) lie in B, and a meanshift
    with a narrow kernel started in B stays in B. So the update must return
    TA, and only a seed at the argmax of L_h does."""
    flows, K, TA, TB, depth, cols = _two_motion_window()
    ow = oracle_lib.OracleWindow(flows, K, S=256, inv_depth_min=0.05, inv_depth_max=1.0,
                                 sigma_t=1e-8, sigma_r=1e-10)
    ow.theta[:] = depth
    ow.poses[0] = TA
    ow.wmap[0][:, :cols] = 0.6
    ow.wmap[0][:, cols:] = 1.0
    R, tv, wts, grp, slot = ow.collect_hypotheses(0, 1)
    L = ow.score(1, R, tv)
    near = lambda i, T: np.abs(R[i] - T[:3, :3]).max() < 1e-9 and np.abs(tv[i] - T[:3, 3]).max() < 1e-9
    best = int(np.argmax(L))
    heavy = next(i for i in range(len(R)) if near(i, TB))       # B's cluster carries the largest weight
    assert near(best, TA) and wts[heavy] == wts.max() == 1.0 and wts[best] < wts.max()
    p6 = np.array([oracle_lib.se3_log(Ri, ti) for Ri, ti in zip(R, tv)])
    _, x_heavy = oracle_lib.meanshift(p6, wts, heavy, 1e-8, 1e-10, 100, 1e-10)
    Rh, th = oracle_lib.se3_exp(x_heavy)
    assert np.abs(th - TB[:3, 3]).max() < 1e-9                  # a wrong seed ends in B
    st, n, L_o, seed, its = ow.pose_update(0, 1)
    assert st == 0 and n == 256 and seed == best
    assert np.abs(L_o - L).max() == 0.0
    assert np.abs(ow.poses[0] - TA).max() < 1e-9
