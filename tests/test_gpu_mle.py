"""GPU parity of the MLE criterion (Eq. 9) against the oracle, teacher-forced
as the MIE tests are: dense pose scores to 1e-5 relative, depth-sweep labels
identical on >= 99.9 % of pixels, and a noiseless window stays at its truth.
The MLE pair term is log2(mu/rho), one SFU logarithm of a quantity that is
never near 1 in the sum's dominant terms, so the MIE tolerances carry over."""
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


def _pair(vd, oracle_lib, w, rng, S=256):
    depth, rig = f32_state(rng, w)
    p = vd.default_params(hyps_per_frame=S, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1], criterion=vd.CRITERION_MLE)
    g = vd.Window(w.flows.astype(np.float32), w.K, p)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), S, depth, rig, w.poses,
                       criterion=1)
    return g, ow, depth, rig


@pytest.mark.parametrize("t", [1, 3])
def test_mle_dense_scores(vd, oracle_lib, scene, t):
    w = scene
    rng = np.random.default_rng(110 + t)
    g, ow, depth, rig = _pair(vd, oracle_lib, w, rng)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    R, tv = f32_hypotheses(rng, w.poses[t - 1][:3, :3], w.poses[t - 1][:3, 3], 64)
    L_gpu = g.score_hypotheses(t, R, tv)
    L_ref = ow.score(t, R, tv)
    rel = np.abs(L_gpu - L_ref) / np.abs(L_ref)
    assert rel.max() < 1e-5, rel.max()
    # and the criterion matters: the MIE scores of the same hypotheses differ
    mie = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), 256, depth, rig, w.poses)
    assert np.abs(mie.score(t, R, tv) - L_ref).max() > 1e-3 * np.abs(L_ref).max()


@pytest.mark.parametrize("k", [0, 1])
def test_mle_depth_sweep(vd, oracle_lib, scene, k):
    w = scene
    rng = np.random.default_rng(150 + k)
    g, ow, depth, rig = _pair(vd, oracle_lib, w, rng)
    q = rng.uniform(0, 1, size=(w.T, w.H, w.W)).astype(np.float32)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=k)
    g.set_buffer(vd.BUF_SMOOTHED, q)
    g.depth_update(k)
    lab_gpu = g.get_buffer(vd.BUF_LABELS, (w.H, w.W), np.uint8)
    _, D_gpu, _ = g.get_pose_depth_rigidness(poses=False, rigidness=False)
    lab_ref = ow.mie_sweep(k, q.astype(np.float64))
    assert np.mean(lab_gpu == lab_ref) >= 0.999
    assert np.mean(np.abs(D_gpu - ow.theta) <= 1e-5 * ow.theta) >= 0.999


def test_mle_noiseless_window_keeps_its_truth(vd):
    """With a pose kernel narrow enough that only the exact P3P solutions carry
    mass (as in the oracle's fixed-point pin), a noiseless window bootstrapped
    at its true T_1 stays at its true poses under MLE."""
    from paper_2104_06789_gb300 import synthetic
    w = synthetic.small_planes(seed=1000, noise=False, nonrigid=False)
    p = vd.default_params(hyps_per_frame=256, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1], criterion=vd.CRITERION_MLE,
                          sigma_t=1e-8, sigma_r=1e-10)
    g = vd.Window(w.flows.astype(np.float32), w.K, p)
    g.bootstrap(w.poses[0])
    g.em_step(2)
    P, _, _ = g.get_pose_depth_rigidness(depth=False, rigidness=False)
    assert np.abs(P[:, :3, :] - w.poses[:, :3, :]).max() < 1e-5
