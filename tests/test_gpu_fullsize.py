"""Parity at the benchmark's full size and launch configuration: the
1242x375, T = 8 driving window with FP16 flows, S = 8192 hypotheses per frame
(the dense scoring's default shape -- 2 hypotheses per thread, three blocks per
SM -- and pixel-chunk count, as bench.py times it), teacher-forced as the small-window tests are.

- dense scores: sampled hypotheses recomputed by the oracle over all 465,750
  pixels, 1e-5 relative; one launch with a full last tile (8192 hypotheses:
  sixteen 512-hypothesis tiles) and two whose last tile is partial (6844: 188
  hypotheses, three groups of 64 scored by two teams of three warps; 6400: 256
  hypotheses scored by two teams of four warps, each team on half of every
  pixel tile);
- per-pixel log-likelihoods (unsmoothed rigidness) at every (t, j): 1e-5
  relative;
- smoothed rigidness (forward-backward) at every (t, j): 2e-5 absolute;
- depth sweep: labels identical on >= 99.9 % of pixels;
- the whole step (bootstrap + 5 EM iterations, as timed by bench.py): the
  poses stay close to the scene's ground truth."""
import numpy as np
import pytest

from tests.helpers import f32_hypotheses, f32_state, oracle_window

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


@pytest.fixture(scope="module")
def drive():
    from paper_2104_06789_gb300 import synthetic
    w = synthetic.driving(seed=3000)
    f16 = np.ascontiguousarray(w.flows.astype(np.float16))
    return w, f16, f16.astype(np.float64)


def _pair(vd, oracle_lib, drive, rng):
    w, f16, f64 = drive
    depth, rig = f32_state(rng, w)
    p = vd.default_params(hyps_per_frame=8192, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1], seed=0, window_id=0)
    g = vd.Window(f16, w.K, p)
    ow = oracle_window(oracle_lib, w, f64, 8192, depth, rig, w.poses)
    return g, ow, depth, rig


@pytest.mark.parametrize("t,n", [(1, 8192), (5, 6844), (7, 6400)])
def test_dense_scores_full_size(vd, oracle_lib, drive, t, n):
    w = drive[0]
    rng = np.random.default_rng(300 + t)
    g, ow, depth, rig = _pair(vd, oracle_lib, drive, rng)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    R, tv = f32_hypotheses(rng, w.poses[t - 1][:3, :3], w.poses[t - 1][:3, 3], n)
    L_gpu = g.score_hypotheses(t, R, tv)
    idx = np.array(sorted({0, 1, 255, 256, 2047, 2048, 4095, 6143, 6144, 6145, 6271, 6338, 6655, 6656, 6843, n - 1} & set(range(n))))
    L_ref = ow.score(t, R[idx], tv[idx])
    rel = np.abs(L_gpu[idx] - L_ref) / np.abs(L_ref)
    assert rel.max() < 1e-5, (rel.max(), idx[np.argmax(rel)])
    g.destroy()


@pytest.mark.parametrize("t", [1, 5, 8])
def test_hypotheses_full_size(vd, oracle_lib, drive, t):
    """Minimal groups drawn over the frame's valid pixels, P3P and the
    collection at S = 8192 in the benchmark's launch shape: exactly S
    hypotheses, the same groups, slots and weights as the oracle, poses to
    1e-9."""
    w = drive[0]
    rng = np.random.default_rng(310 + t)
    g, ow, depth, rig = _pair(vd, oracle_lib, drive, rng)
    rig = (0.5 + 0.5 * rig).astype(np.float32)
    ow.wmap[:] = rig.astype(np.float64)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=1)
    g.pose_update(1, t)
    hg = g.hypotheses()
    R, tv, wts, grp, slot = ow.collect_hypotheses(1, t)
    assert len(R) == 8192 and len(hg["R"]) == 8192
    assert np.array_equal(hg["group"], grp) and np.array_equal(hg["slot"], slot)
    assert np.array_equal(hg["weight"], wts)
    # translations to 1e-9 relative to their size: spurious roots of far,
    # thin triangles reach hundreds of metres, and P3P magnifies the FP64
    # rounding of its inputs there (the two sides form K^-1 [x y 1] with a
    # reciprocal and with a division)
    assert np.abs(hg["R"] - R).max() < 1e-9
    dt = np.linalg.norm(hg["t"] - tv, axis=1) / np.maximum(np.linalg.norm(tv, axis=1), 1.0)
    assert dt.max() < 1e-9, dt.max()
    g.destroy()


def test_rigidness_full_size(vd, oracle_lib, drive):
    w = drive[0]
    rng = np.random.default_rng(320)
    g, ow, depth, rig = _pair(vd, oracle_lib, drive, rng)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    g.rigidness_update()
    _, _, W_gpu = g.get_pose_depth_rigidness(poses=False, depth=False)
    W_ref = ow.emissions()
    ell_ref = np.log(W_ref)
    err = np.abs(np.log(W_gpu.astype(np.float64)) - ell_ref)
    assert np.all(err <= 1e-5 * np.abs(ell_ref) + 2.0 ** -23), err.max()
    # smoothed (E-step) along rows, as the first iteration's forward-backward runs
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    g.rigidness_smooth(0)
    q_gpu = g.get_buffer(vd.BUF_SMOOTHED, (w.T, w.H, w.W), np.float32)
    q_ref = ow.smooth(0, W_ref)
    assert np.abs(q_gpu - q_ref).max() < 2e-5
    g.destroy()


def test_depth_sweep_full_size(vd, oracle_lib, drive):
    w = drive[0]
    rng = np.random.default_rng(330)
    g, ow, depth, rig = _pair(vd, oracle_lib, drive, rng)
    q = rng.uniform(0, 1, size=(w.T, w.H, w.W)).astype(np.float32)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=1)
    g.set_buffer(vd.BUF_SMOOTHED, q)
    g.depth_update(1)
    lab_gpu = g.get_buffer(vd.BUF_LABELS, (w.H, w.W), np.uint8)
    _, D_gpu, _ = g.get_pose_depth_rigidness(poses=False, rigidness=False)
    lab_ref = ow.mie_sweep(1, q.astype(np.float64))
    assert np.mean(lab_gpu == lab_ref) >= 0.999
    assert np.mean(np.abs(D_gpu - ow.theta) <= 1e-5 * ow.theta) >= 0.999
    g.destroy()


def test_em_step_full_size_tracks_the_ground_truth(vd, drive):
    w, f16, _ = drive
    p = vd.default_params(hyps_per_frame=8192, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1], seed=0, window_id=0)
    g = vd.Window(f16, w.K, p)
    g.bootstrap(w.poses[0])
    g.em_step(5)
    P, D, Wm = g.get_pose_depth_rigidness()
    dt = np.linalg.norm(P[:, :3, 3] - w.poses[:, :3, 3], axis=1)
    cosang = (np.einsum("tij,tij->t", P[:, :3, :3], w.poses[:, :3, :3]) - 1.0) / 2.0
    ang = np.degrees(np.arccos(np.clip(cosang, -1.0, 1.0)))
    print("translation error per frame (m)", dt, "rotation error (deg)", ang)
    assert np.all(np.isfinite(P)) and np.all(np.isfinite(D)) and np.all((Wm >= 0) & (Wm <= 1))
    assert dt.max() < 0.05 and ang.max() < 0.2, (dt, ang)
    g.destroy()
