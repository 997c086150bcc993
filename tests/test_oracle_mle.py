"""Pins of the oracle's MLE criterion (Eq. 9): its per-(t, j) term against
scipy's Fisk density, its convention for invalid terms, the sweep's
monotonicity and the noiseless fixed point."""
import numpy as np
import pytest
from scipy import stats

from conftest import fronto_parallel_window
from paper_2104_06789_gb300 import synthetic


def test_mle_term_is_the_log_density_ratio(oracle_lib):
    w = synthetic.small_planes(seed=1001)
    ow = oracle_lib.OracleWindow(w.flows, w.K, criterion=1)
    ow.poses[:] = w.poses
    rng = np.random.default_rng(0)
    p = oracle_lib.PAPER_DEFAULTS
    checked = 0
    for _ in range(60):
        t = int(rng.integers(1, w.T + 1))
        j = int(rng.integers(0, w.W * w.H))
        depth = float(w.depth0.flat[j] * rng.uniform(0.8, 1.2))
        v, diag = ow.frame_eval(t, j, depth)
        crit = ow.frame_crit(t, j, depth)
        if v < 2:                       # no observation at pi_{t-1}, or behind camera t: rho := mu
            assert crit == 0.0
            continue
        res, vob = diag[0:2], diag[4:6]
        n = np.hypot(*vob)
        alpha = p["a1"] * np.exp(p["a2"] * n)
        beta = max(p["b1"] * n + p["b2"], p["beta_min"])
        x = np.clip(res @ res, p["x_min"], p["x_max"])
        x_mu = np.clip(p["lambda_"] ** 2 * n * n, p["x_min"], p["x_max"])
        ref = stats.fisk.logpdf(x, beta, scale=alpha) - stats.fisk.logpdf(x_mu, beta, scale=alpha)
        assert crit == pytest.approx(ref, rel=1e-10, abs=1e-10)
        checked += 1
    assert checked > 30


def test_mie_and_mle_differ_only_in_the_criterion(oracle_lib):
    w = synthetic.small_planes(seed=1001)
    a = oracle_lib.OracleWindow(w.flows, w.K, criterion=0)
    b = oracle_lib.OracleWindow(w.flows, w.K, criterion=1)
    for o in (a, b):
        o.poses[:] = w.poses
    t = 2
    for j in range(5000, w.W * w.H):                      # a (t, j) with an observation in front of camera t
        d = float(w.depth0.flat[j])
        va, da = a.frame_eval(t, j, d)
        if va == 2:
            break
    vb, db = b.frame_eval(t, j, d)
    assert va == vb == 2 and np.array_equal(da, db)      # the geometry and densities are shared
    log_rho, log_mu = da[6], da[7]
    assert a.frame_crit(t, j, d) == pytest.approx(-np.logaddexp(0.0, log_mu - log_rho), rel=1e-12)
    assert b.frame_crit(t, j, d) == pytest.approx(log_rho - log_mu, rel=1e-12)
    # the E-step posterior does not depend on the criterion
    assert np.array_equal(a.emissions(), b.emissions())


def test_mle_sweep_monotone_and_fixed_point(oracle_lib):
    flows, K, poses, depth = fronto_parallel_window(T=3)
    ow = oracle_lib.OracleWindow(flows, K, S=8, inv_depth_min=0.05, inv_depth_max=1.0, criterion=1)
    ow.theta[:] = depth
    ow.poses[:] = poses
    q = np.ones((3,) + depth.shape)
    labels = ow.mie_sweep(0, q)
    assert np.all(labels == 0)
    assert np.array_equal(ow.theta, depth)
    rng = np.random.default_rng(1)
    start = depth * rng.uniform(0.7, 1.4, size=depth.shape)
    for k in range(4):
        ow.theta[:] = start
        before = np.array([ow.mie_score(q, j, start.flat[j]) for j in range(depth.size)])
        ow.mie_sweep(k, q)
        after = np.array([ow.mie_score(q, j, ow.theta.flat[j]) for j in range(depth.size)])
        assert np.all(after >= before)


def test_mle_full_loop_noiseless_fixed_point(oracle_lib):
    flows, K, poses, depth = fronto_parallel_window(W=24, H=18, T=3)
    ow = oracle_lib.OracleWindow(flows, K, S=32, inv_depth_min=0.05, inv_depth_max=1.0,
                                 sigma_t=1e-8, sigma_r=1e-10, criterion=1)
    ow.bootstrap(poses[0])
    st = ow.run(0, 2)
    assert st == 0
    assert np.abs(ow.poses - poses).max() < 1e-9
    assert np.max(np.abs(ow.theta - depth)) < 1e-12
