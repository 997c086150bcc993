"""The epipolar bootstrap (LMedS essential matrix of X_1) through the C ABI
against the oracle.

Per sample: validity identical, the FP64 essential matrix to 1e-8 (same eight
correspondences, different null-space and projection methods), the FP32 median
Sampson error to 2e-5 relative (an order statistic moves by no more than the
largest perturbation of the values, ~1e-6 relative for the cancellation-free
FP32 form). The winner is judged by the oracle: its oracle score is within
2e-5 of the smallest. The refined T_1 is the least-squares fit over the
winner's inliers, which are decided by the Sampson error at a threshold: in
FP32 on the GPU, in FP64 in the oracle, so a few borderline pixels flip; the
two smallest eigenvalues of the fit's normal matrix are 0.0025 and 0.4 here,
so each flip moves the fit by ~1e-5, and on noisy windows the inlier counts
are compared to 0.1 % and T_1 to 1e-4 rad (rotation) and 1e-3 (unit
translation). On noiseless windows
both sides recover the generating pose; the GPU's reweighted fit solves the
normal equations A^T A (the oracle works on A), which squares the condition
number, so there the bound is 1e-7 (matrix entries, not an arccos angle, whose
resolution near zero is ~1.5e-8).
"""
import numpy as np
import pytest

import oracle
from paper_2104_06789_gb300 import synthetic

from helpers import rotation_angle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


def _windows(vd, w, flows, **kw):
    p = vd.default_params(inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1],
                          hyps_per_frame=64, **kw)
    g = vd.Window(flows.astype(np.float32), w.K, p)
    ow = oracle.OracleWindow(flows.astype(np.float32).astype(np.float64), w.K, inv_depth_min=w.inv_depth_range[0],
                             inv_depth_max=w.inv_depth_range[1], **kw)
    return g, ow


def _sign_aligned(a, b):
    a = a / np.linalg.norm(a)
    b = b / np.linalg.norm(b)
    return a * np.sign(np.sum(a * b)), b


@pytest.mark.parametrize("nonrigid", [False, True])
def test_noiseless_window_recovers_the_generating_pose(vd, nonrigid):
    w = synthetic.small_planes(seed=1000, noise=False, nonrigid=nonrigid)
    g, ow = _windows(vd, w, w.flows)
    base = float(np.linalg.norm(w.poses[0][:3, 3]))
    T1 = g.bootstrap_epipolar(64, base)
    assert np.abs(T1[:3, :3] - w.poses[0][:3, :3]).max() < 1e-7
    assert np.abs(T1[:3, 3] - w.poses[0][:3, 3]).max() < 1e-7 * base
    _, D, Wm = g.get_pose_depth_rigidness(poses=False)
    ow.bootstrap(T1)
    assert np.allclose(D, ow.theta, rtol=1e-6)
    assert np.all(Wm == 1.0)
    g.destroy()


@pytest.mark.parametrize("seed", [3001, 3003])
def test_samples_medians_and_pose_match_the_oracle(vd, seed):
    w = synthetic.driving(seed=seed, W=414, H=125, f=239.3, T=2)
    flows = w.flows.astype(np.float16).astype(np.float32)      # FP16-representable, as the driving window stores them
    g, ow = _windows(vd, w, flows)
    M = 160
    T1 = g.bootstrap_epipolar(M, 1.0)
    r = g.epipolar_results()
    st, T1_or, scores, m_or, c_or = ow.epipolar_bootstrap(M, 1.0)
    assert st == 0
    n_cmp = 0
    for m in range(M):
        ok, E_or, _ = ow.epi_sample(m)
        assert bool(ok) == bool(r["valid"][m]), m
        if not ok:
            assert np.isinf(r["medians"][m])
            continue
        a, b = _sign_aligned(r["E"][m], E_or)
        assert np.abs(a - b).max() < 1e-8, m
        assert r["medians"][m] == pytest.approx(scores[m], rel=2e-5), m
        n_cmp += 1
    assert n_cmp >= 8           # many samples hold a pixel whose target leaves the image (fast forward motion)
    assert scores[r["chosen"]] <= (1 + 2e-5) * scores.min()
    assert r["n_valid"] == sum(1 for j in range(w.W * w.H) if _valid(flows[0], j, w.W, w.H))
    n_or, _, _ = ow.epi_refine(ow.epi_sample(r["chosen"])[1], scores[r["chosen"]])
    assert abs(r["n_inliers"] - n_or) <= 1e-3 * n_or
    assert rotation_angle(T1[:3, :3], T1_or[:3, :3]) < 1e-4
    assert np.abs(T1[:3, 3] - T1_or[:3, 3]).max() < 1e-3
    # the triangulated depth follows the GPU's own T_1 exactly
    _, D, _ = g.get_pose_depth_rigidness(poses=False, rigidness=False)
    ref = oracle.OracleWindow(flows.astype(np.float64), w.K, inv_depth_min=w.inv_depth_range[0],
                              inv_depth_max=w.inv_depth_range[1])
    ref.bootstrap(T1)
    assert np.allclose(D, ref.theta, rtol=1e-6)
    g.destroy()


def _valid(f0, j, W, H):
    x, y = j % W, j // W
    u, v = x + float(f0[y, x, 0]), y + float(f0[y, x, 1])
    return 0.0 <= u <= W - 1 and 0.0 <= v <= H - 1


def test_no_valid_pixel_is_degenerate_and_leaves_the_window_unbootstrapped(vd):
    w = synthetic.small_planes(seed=1000)
    flows = np.full_like(w.flows, 5000.0)
    g, _ = _windows(vd, w, flows)
    with pytest.raises(vd.VoldorError) as ei:
        g.bootstrap_epipolar(16, 1.0)
    assert ei.value.status == vd.ERR_DEGENERATE
    assert vd.lib().voldor_em_step(g._h, 1) == vd.ERR_NOT_BOOTSTRAPPED
    g.destroy()


def test_invalid_arguments(vd):
    w = synthetic.small_planes(seed=1000)
    g, _ = _windows(vd, w, w.flows)
    L = vd.lib()
    for n, b in [(0, 1.0), (vd.EPI_MAX_SAMPLES + 1, 1.0), (8, 0.0), (8, float("nan")), (8, -1.0)]:
        assert L.voldor_bootstrap_epipolar(g._h, n, b, None) == vd.ERR_INVALID_ARG
    g.destroy()


def test_bootstrap_mode_epipolar_equals_the_epipolar_call(vd):
    """voldor_bootstrap(ctx, VOLDOR_BOOT_EPIPOLAR, NULL) is the epipolar
    bootstrap with 512 samples and |t_1| = 1: same poses, depth and state."""
    w = synthetic.driving(seed=3001, W=414, H=125, f=239.3, T=3)
    p = vd.default_params(inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1],
                          hyps_per_frame=64)
    a = vd.Window(w.flows.astype(np.float32), w.K, p)
    b = vd.Window(w.flows.astype(np.float32), w.K, p)
    T1 = a.bootstrap_epipolar(512, 1.0)
    assert vd.lib().voldor_bootstrap(b._h, vd.BOOT_EPIPOLAR, None) == vd.OK
    Pa, Da, Wa = a.get_pose_depth_rigidness()
    Pb, Db, Wb = b.get_pose_depth_rigidness()
    assert np.array_equal(Pa, Pb) and np.array_equal(Da, Db) and np.array_equal(Wa, Wb)
    assert np.linalg.norm(T1[:3, 3]) == pytest.approx(1.0, rel=1e-12)
    assert vd.lib().voldor_bootstrap(b._h, 1, None) == vd.ERR_INVALID_ARG      # the learned mode needs the network
    a.destroy()
    b.destroy()
