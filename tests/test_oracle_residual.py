"""Pins of the oracle's Gaussian residual model (the alternative model of the
ablation study, Sec. 6.3), checked against scipy: the squared EPE of an
isotropic 2-D normal residual is chi-square with 2 degrees of freedom scaled
by sigma^2; the variance is matched to the Fisk model by the median (the
Fisk median is alpha); and the window's per-(t, j) terms use that density for
both rho and mu (Eq. 7), under MIE and MLE."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from paper_2104_06789_gb300 import synthetic


def test_gauss_logpdf_is_the_chi2_density_of_a_2d_normal(oracle_lib):
    for alpha in (0.01, 0.3, 2.0, 40.0):
        sigma2 = alpha / (2.0 * math.log(2.0))
        for x in (1e-6, 0.01, alpha, 3.7 * alpha, 50.0):
            ref = stats.chi2(df=2, scale=sigma2).logpdf(x)
            assert oracle_lib.gauss_logpdf(x, math.log(alpha)) == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_gauss_median_matches_the_fisk_median(oracle_lib):
    for alpha in (0.05, 1.0, 7.5):
        f = lambda x: math.exp(oracle_lib.gauss_logpdf(x, math.log(alpha)))
        total, _ = integrate.quad(f, 0, np.inf)
        below, _ = integrate.quad(f, 0, alpha)
        assert total == pytest.approx(1.0, rel=1e-9)
        assert below == pytest.approx(0.5, rel=1e-9)
        # and alpha is the Fisk model's median for any shape
        assert stats.fisk(c=0.7, scale=alpha).median() == pytest.approx(alpha, rel=1e-12)


@pytest.mark.parametrize("criterion", [0, 1])
def test_window_terms_use_the_gaussian_density(oracle_lib, criterion):
    w = synthetic.small_planes(seed=1001)
    ow = oracle_lib.OracleWindow(w.flows, w.K, criterion=criterion, residual=1)
    ow.poses[:] = w.poses
    fisk = oracle_lib.OracleWindow(w.flows, w.K, criterion=criterion, residual=0)
    fisk.poses[:] = w.poses
    rng = np.random.default_rng(3)
    p = oracle_lib.PAPER_DEFAULTS
    checked = 0
    for _ in range(60):
        t = int(rng.integers(1, w.T + 1))
        j = int(rng.integers(0, w.W * w.H))
        depth = float(w.depth0.flat[j] * rng.uniform(0.8, 1.2))
        v, diag = ow.frame_eval(t, j, depth)
        crit = ow.frame_crit(t, j, depth)
        if v < 2:                       # rho := mu
            assert crit == (0.0 if criterion else pytest.approx(math.log(0.5)))
            continue
        res, vob = diag[0:2], diag[4:6]
        n = np.hypot(*vob)
        alpha = p["a1"] * np.exp(p["a2"] * n)
        sigma2 = alpha / (2.0 * math.log(2.0))
        x = np.clip(res @ res, p["x_min"], p["x_max"])
        x_mu = np.clip(p["lambda_"] ** 2 * n * n, p["x_min"], p["x_max"])
        log_rho = stats.chi2(df=2, scale=sigma2).logpdf(x)
        log_mu = stats.chi2(df=2, scale=sigma2).logpdf(x_mu)
        ref = log_rho - log_mu if criterion else -np.logaddexp(0.0, log_mu - log_rho)
        assert crit == pytest.approx(ref, rel=1e-10, abs=1e-10)
        # the geometry is shared with the Fisk window; only the densities differ
        vf, df = fisk.frame_eval(t, j, depth)
        assert vf == v and np.array_equal(df[:6], diag[:6])
        checked += 1
    assert checked > 30
