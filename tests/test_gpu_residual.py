"""GPU parity of the Gaussian residual model (the ablation study's
alternative to the Fisk model, Sec. 6.3) against the oracle, teacher-forced
as the Fisk tests are: dense pose scores to 1e-5 relative under MIE and MLE,
per-pixel log-likelihoods to 1e-5 relative (where they are representable: an
outlier's Gaussian log-likelihood reaches -1e4 and its W underflows to 0 on
both sides), depth-sweep labels identical on >= 99.9 % of pixels, and a
noiseless window stays at its truth."""
import numpy as np
import pytest

from tests.helpers import f32_hypotheses, f32_state, oracle_window, small_window

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


@pytest.fixture(scope="module")
def scene():
    return small_window(seed=1000)


def _pair(vd, oracle_lib, w, rng, criterion, S=256):
    depth, rig = f32_state(rng, w)
    p = vd.default_params(hyps_per_frame=S, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1], criterion=criterion,
                          residual=vd.RESIDUAL_GAUSSIAN)
    g = vd.Window(w.flows.astype(np.float32), w.K, p)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), S, depth, rig, w.poses,
                       criterion=criterion, residual=1)
    return g, ow, depth, rig


@pytest.mark.parametrize("criterion", [0, 1])
@pytest.mark.parametrize("t", [1, 3])
def test_gaussian_dense_scores(vd, oracle_lib, scene, t, criterion):
    w = scene
    rng = np.random.default_rng(210 + t + 10 * criterion)
    g, ow, depth, rig = _pair(vd, oracle_lib, w, rng, criterion)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    R, tv = f32_hypotheses(rng, w.poses[t - 1][:3, :3], w.poses[t - 1][:3, 3], 64)
    L_gpu = g.score_hypotheses(t, R, tv)
    L_ref = ow.score(t, R, tv)
    rel = np.abs(L_gpu - L_ref) / np.abs(L_ref)
    assert rel.max() < 1e-5, rel.max()
    # and the model matters: the Fisk scores of the same hypotheses differ
    fisk = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), 256, depth, rig, w.poses,
                         criterion=criterion)
    assert np.abs(fisk.score(t, R, tv) - L_ref).max() > 1e-3 * np.abs(L_ref).max()


def test_gaussian_unsmoothed_rigidness(vd, oracle_lib, scene):
    w = scene
    rng = np.random.default_rng(240)
    g, ow, depth, rig = _pair(vd, oracle_lib, w, rng, 0)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    g.rigidness_update()
    _, _, W_gpu = g.get_pose_depth_rigidness(poses=False, depth=False)
    W_ref = ow.emissions()
    ok = W_ref > 1e-30
    assert ok.mean() > 0.5
    ell_ref = np.log(W_ref[ok])
    err = np.abs(np.log(W_gpu[ok].astype(np.float64)) - ell_ref)
    assert np.all(err <= 1e-5 * np.abs(ell_ref) + 2.0 ** -23), err.max()
    assert np.all(W_gpu[~ok] <= 1e-29)


@pytest.mark.parametrize("criterion", [0, 1])
def test_gaussian_depth_sweep(vd, oracle_lib, scene, criterion):
    w = scene
    rng = np.random.default_rng(250 + criterion)
    g, ow, depth, rig = _pair(vd, oracle_lib, w, rng, criterion)
    q = rng.uniform(0, 1, size=(w.T, w.H, w.W)).astype(np.float32)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=1)
    g.set_buffer(vd.BUF_SMOOTHED, q)
    g.depth_update(1)
    lab_gpu = g.get_buffer(vd.BUF_LABELS, (w.H, w.W), np.uint8)
    _, D_gpu, _ = g.get_pose_depth_rigidness(poses=False, rigidness=False)
    lab_ref = ow.mie_sweep(1, q.astype(np.float64))
    assert np.mean(lab_gpu == lab_ref) >= 0.999
    assert np.mean(np.abs(D_gpu - ow.theta) <= 1e-5 * ow.theta) >= 0.999


def test_gaussian_noiseless_window_keeps_its_truth(vd):
    """A fronto-parallel plane under translation (constant flows, so bilinear
    sampling is exact and no pixel is an outlier) bootstrapped at its true
    T_1 stays at its true poses under the Gaussian model. (On scenes with
    depth edges the noiseless window is not a fixed point of this model: the
    few pixels whose bilinear flow sample straddles an edge are outliers, and
    the Gaussian model's MIE term grows linearly in their squared residual
    instead of saturating as the Fisk model's does.)"""
    from conftest import fronto_parallel_window
    flows, K, poses, depth = fronto_parallel_window(W=48, H=36, T=3, f=40.0)
    p = vd.default_params(hyps_per_frame=256, inv_depth_min=1 / 40.0, inv_depth_max=1.0,
                          residual=vd.RESIDUAL_GAUSSIAN, sigma_t=1e-8, sigma_r=1e-10)
    g = vd.Window(flows.astype(np.float32), K, p)
    g.bootstrap(poses[0])
    g.em_step(2)
    P, D, _ = g.get_pose_depth_rigidness(rigidness=False)
    assert np.abs(P[:, :3, :] - poses[:, :3, :]).max() < 1e-5
    assert np.abs(D - depth).max() < 1e-4 * depth.max()
