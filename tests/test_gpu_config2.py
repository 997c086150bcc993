"""Parity on the handheld window at its full size (640x480, f = 525, T = 5,
FP32 flows, S = 4096 hypotheses per frame), teacher-forced like the stage
tests (both sides get the same FP32-representable state):

- dense scores of sampled hypotheses against the oracle over all 307,200
  pixels, 1e-5 relative; one launch with full hypothesis tiles (4096) and one
  whose last tile is partial (3000);
- minimal groups, P3P and the collection of exactly S hypotheses: the same
  groups, slots and weights as the oracle, poses to 1e-9;
- per-pixel log-likelihoods (unsmoothed rigidness) at every (t, j): 1e-5
  relative plus the FP32 storage of W; smoothed rigidness along columns: 2e-5;
- depth sweep (right to left): labels identical on >= 99.9 % of pixels;
- bootstrap + 5 EM iterations: finite outputs, and every frame's pose closer
  to the scene's truth than the bootstrap's (T_t = T_1 for every t) was."""
import numpy as np
import pytest

from tests.helpers import f32_hypotheses, f32_state, oracle_window

pytestmark = pytest.mark.gpu

S = 4096


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


@pytest.fixture(scope="module")
def hand():
    from paper_2104_06789_gb300 import synthetic
    w = synthetic.handheld(seed=2000)
    f32 = np.ascontiguousarray(w.flows.astype(np.float32))
    return w, f32, f32.astype(np.float64)


def _pair(vd, oracle_lib, hand, rng):
    w, f32, f64 = hand
    depth, rig = f32_state(rng, w)
    p = vd.default_params(hyps_per_frame=S, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1], seed=0, window_id=0)
    g = vd.Window(f32, w.K, p)
    ow = oracle_window(oracle_lib, w, f64, S, depth, rig, w.poses)
    return g, ow, depth, rig


@pytest.mark.parametrize("t,n", [(1, 4096), (5, 3000)])
def test_dense_scores_config2(vd, oracle_lib, hand, t, n):
    w = hand[0]
    rng = np.random.default_rng(400 + t)
    g, ow, depth, rig = _pair(vd, oracle_lib, hand, rng)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    R, tv = f32_hypotheses(rng, w.poses[t - 1][:3, :3], w.poses[t - 1][:3, 3], n)
    L_gpu = g.score_hypotheses(t, R, tv)
    idx = np.array(sorted({0, 1, 255, 256, 1023, 1024, 2047, 2048, 2943, 2944, 2999, n - 1} & set(range(n))))
    L_ref = ow.score(t, R[idx], tv[idx])
    rel = np.abs(L_gpu[idx] - L_ref) / np.abs(L_ref)
    assert rel.max() < 1e-5, (rel.max(), idx[np.argmax(rel)])
    g.destroy()


@pytest.mark.parametrize("t", [1, 3, 5])
def test_hypotheses_config2(vd, oracle_lib, hand, t):
    w = hand[0]
    rng = np.random.default_rng(410 + t)
    g, ow, depth, rig = _pair(vd, oracle_lib, hand, rng)
    rig = (0.5 + 0.5 * rig).astype(np.float32)
    ow.wmap[:] = rig.astype(np.float64)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=1)
    g.pose_update(1, t)
    hg = g.hypotheses()
    R, tv, wts, grp, slot = ow.collect_hypotheses(1, t)
    assert len(R) == S and len(hg["R"]) == S
    assert np.array_equal(hg["group"], grp) and np.array_equal(hg["slot"], slot)
    assert np.array_equal(hg["weight"], wts)
    assert np.abs(hg["R"] - R).max() < 1e-9
    dt = np.linalg.norm(hg["t"] - tv, axis=1) / np.maximum(np.linalg.norm(tv, axis=1), 1.0)
    assert dt.max() < 1e-9, dt.max()
    g.destroy()


def test_rigidness_config2(vd, oracle_lib, hand):
    w = hand[0]
    rng = np.random.default_rng(420)
    g, ow, depth, rig = _pair(vd, oracle_lib, hand, rng)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=1)
    g.rigidness_update()
    _, _, W_gpu = g.get_pose_depth_rigidness(poses=False, depth=False)
    W_ref = ow.emissions()
    ell_ref = np.log(W_ref)
    err = np.abs(np.log(W_gpu.astype(np.float64)) - ell_ref)
    assert np.all(err <= 1e-5 * np.abs(ell_ref) + 2.0 ** -23), err.max()
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=1)
    g.rigidness_smooth(1)                              # columns, as iteration 1 smooths
    q_gpu = g.get_buffer(vd.BUF_SMOOTHED, (w.T, w.H, w.W), np.float32)
    q_ref = ow.smooth(1, W_ref)
    assert np.abs(q_gpu - q_ref).max() < 2e-5
    g.destroy()


def test_depth_sweep_config2(vd, oracle_lib, hand):
    w = hand[0]
    rng = np.random.default_rng(430)
    g, ow, depth, rig = _pair(vd, oracle_lib, hand, rng)
    q = rng.uniform(0, 1, size=(w.T, w.H, w.W)).astype(np.float32)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=2)
    g.set_buffer(vd.BUF_SMOOTHED, q)
    g.depth_update(2)
    lab_gpu = g.get_buffer(vd.BUF_LABELS, (w.H, w.W), np.uint8)
    _, D_gpu, _ = g.get_pose_depth_rigidness(poses=False, rigidness=False)
    lab_ref = ow.mie_sweep(2, q.astype(np.float64))
    assert np.mean(lab_gpu == lab_ref) >= 0.999
    assert np.mean(np.abs(D_gpu - ow.theta) <= 1e-5 * ow.theta) >= 0.999
    g.destroy()


def test_em_step_config2_improves_on_its_start(vd, hand):
    w, f32, _ = hand
    p = vd.default_params(hyps_per_frame=S, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1], seed=0, window_id=0)
    g = vd.Window(f32, w.K, p)
    g.bootstrap(w.poses[0])
    P0, _, _ = g.get_pose_depth_rigidness(depth=False, rigidness=False)
    g.em_step(5)
    P, D, Wm = g.get_pose_depth_rigidness()
    assert np.all(np.isfinite(P)) and np.all(np.isfinite(D)) and np.all((Wm >= 0) & (Wm <= 1))
    e0 = np.linalg.norm(P0[:, :3, 3] - w.poses[:, :3, 3], axis=1)
    e = np.linalg.norm(P[:, :3, 3] - w.poses[:, :3, 3], axis=1)
    print("translation error per frame (m): bootstrap", e0, "after 5 iterations", e)
    assert np.all(e[1:] < e0[1:]), (e0, e)
    g.destroy()
