"""GPU parity: each CUDA stage against the FP64 oracle, teacher-forced (both
sides get the same FP32-representable state and run one sub-step).

Tolerances (derived in the design notes from the FP32 arithmetic):
  - dense scores L_h: 1e-5 relative;
  - per-pixel log-likelihood terms and rigidness maps: absolute 2e-5 on
    quantities in [0, 1], relative 1e-5 on sums;
  - P3P hypotheses: identical group indices and slots, poses to 1e-9;
  - pose after meanshift: 1e-6 rad and 1e-6 relative translation;
  - depth candidates: identical labels on >= 99.9% of pixels.
"""
import numpy as np
import pytest

from tests.helpers import f32_hypotheses, f32_state, oracle_window, pose_close, small_window

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


@pytest.fixture(scope="module")
def scene():
    return small_window(seed=1000)


def _gpu_window(vd, w, S=256, flows=None, **kw):
    flows = w.flows.astype(np.float32) if flows is None else flows
    p = vd.default_params(hyps_per_frame=S, inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1], **kw)
    return vd.Window(flows, w.K, p)


def test_bootstrap(vd, oracle_lib, scene):
    w = scene
    g = _gpu_window(vd, w)
    g.bootstrap(w.poses[0])
    P, D, Wm = g.get_pose_depth_rigidness()
    ow = oracle_lib.OracleWindow(w.flows.astype(np.float32).astype(np.float64), w.K, S=8,
                                 inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1])
    ow.bootstrap(w.poses[0])
    assert np.all(Wm == 1.0)
    assert np.allclose(P, np.broadcast_to(w.poses[0], P.shape), rtol=0, atol=0)
    rel = np.abs(D - ow.theta) / ow.theta
    assert rel.max() < 1e-6          # FP64 triangulation, FP32 storage


# hypothesis counts: 1, 64 and 200 leave one partial tile that the block's
# warps split into 8, 8 and 2 teams over the pixels; 1100 is a full
# 1024-hypothesis tile plus a ragged 76-hypothesis one
@pytest.mark.parametrize("t,n", [(1, 1), (1, 64), (2, 64), (3, 64), (1, 200), (2, 1100), (3, 1100)])
def test_dense_scores(vd, oracle_lib, scene, t, n):
    w = scene
    rng = np.random.default_rng(10 + t)
    depth, rig = f32_state(rng, w)
    g = _gpu_window(vd, w, S=max(256, n))
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), 256, depth, rig, w.poses)
    R, tv = f32_hypotheses(rng, w.poses[t - 1][:3, :3], w.poses[t - 1][:3, 3], n)
    L_gpu = g.score_hypotheses(t, R, tv)
    L_ref = ow.score(t, R, tv)
    rel = np.abs(L_gpu - L_ref) / np.abs(L_ref)
    assert rel.max() < 1e-5, rel.max()


# every dense-scoring shape the autotuner can pick (2, 4 or 8 hypotheses per
# thread: 3, 2 or 1 blocks per SM), with ragged pixel-chunk counts and a
# partial last hypothesis tile
@pytest.mark.parametrize("hpt,chunks,n", [(2, 7, 700), (2, 13, 1100), (4, 7, 1100), (8, 5, 2100)])
def test_dense_scores_every_shape(vd, oracle_lib, scene, hpt, chunks, n):
    w = scene
    t = 2
    rng = np.random.default_rng(60 + hpt + n)
    depth, rig = f32_state(rng, w)
    g = _gpu_window(vd, w, S=max(256, n))
    g.set_score_shape(hpt, chunks)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), 256, depth, rig, w.poses)
    R, tv = f32_hypotheses(rng, w.poses[t - 1][:3, :3], w.poses[t - 1][:3, 3], n)
    L_gpu = g.score_hypotheses(t, R, tv)
    L_ref = ow.score(t, R, tv)
    rel = np.abs(L_gpu - L_ref) / np.abs(L_ref)
    assert rel.max() < 1e-5, rel.max()
    g.destroy()


# tiny images (108 and 231 pixels): the pixel chunks hold one or a few
# records, so pixel tiles of a single pixel (the pipelined pixel loop's first
# and last stage only) and warp teams with an empty share of a tile occur
@pytest.mark.parametrize("shape,n", [((12, 9), 1), ((12, 9), 300), ((33, 7), 64), ((33, 7), 1100)])
def test_dense_scores_tiny_images(vd, oracle_lib, shape, n):
    W, H = shape
    w = small_window(seed=1100 + W, W=W, H=H, f=W * 0.75)
    rng = np.random.default_rng(W + n)
    depth, rig = f32_state(rng, w)
    g = _gpu_window(vd, w, S=max(256, n))
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), 256, depth, rig, w.poses)
    R, tv = f32_hypotheses(rng, w.poses[0][:3, :3], w.poses[0][:3, 3], n)
    L_gpu = g.score_hypotheses(1, R, tv)
    L_ref = ow.score(1, R, tv)
    rel = np.abs(L_gpu - L_ref) / np.abs(L_ref)
    assert rel.max() < 1e-5, rel.max()
    g.destroy()


@pytest.mark.parametrize("t", [1, 3])
def test_pose_update(vd, oracle_lib, scene, t):
    w = scene
    rng = np.random.default_rng(20 + t)
    depth, rig = f32_state(rng, w)
    rig = (0.5 + 0.5 * rig).astype(np.float32)
    g = _gpu_window(vd, w)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=1)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), 256, depth, rig, w.poses)
    k = 1
    g.pose_update(k, t)
    hg = g.hypotheses()
    R, tv, wts, grp, slot = ow.collect_hypotheses(k, t)
    assert len(R) == 256 and len(hg["R"]) == len(R)        # exactly S
    assert grp[-1] < 4 * 256
    assert np.array_equal(hg["group"], grp) and np.array_equal(hg["slot"], slot)
    assert np.array_equal(hg["weight"], wts)
    assert np.abs(hg["R"] - R).max() < 1e-9 and np.abs(hg["t"] - tv).max() < 1e-9
    # scores of the FP32 scoring form, scored by the oracle
    f32 = g.get_buffer(vd.BUF_HYPS_F32, (256, 12), np.float32)[:len(R)].astype(np.float64)
    Rf = np.eye(3) + f32[:, :9].reshape(-1, 3, 3)
    L_ref = ow.score(t, Rf, f32[:, 9:])
    rel = np.abs(hg["L"] - L_ref) / np.abs(L_ref)
    assert rel.max() < 1e-5
    # the pose: oracle's full update on the same state
    st, n, L_o, seed_o, its = ow.pose_update(k, t)
    P_gpu, _, _ = g.get_pose_depth_rigidness(depth=False, rigidness=False)
    ok, ang, dt = pose_close(P_gpu[t - 1], ow.poses[t - 1])
    assert ok, (ang, dt, hg["seed"], seed_o)


@pytest.mark.parametrize("k", [0, 1])
def test_smoothed_rigidness(vd, oracle_lib, scene, k):
    w = scene
    rng = np.random.default_rng(30 + k)
    depth, rig = f32_state(rng, w)
    g = _gpu_window(vd, w)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=k)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), 256, depth, rig, w.poses)
    g.rigidness_smooth(k)
    q_gpu = g.get_buffer(vd.BUF_SMOOTHED, (w.T, w.H, w.W), np.float32)
    em = ow.emissions()
    q_ref = ow.smooth(0 if k % 2 == 0 else 1, em)
    assert np.abs(q_gpu - q_ref).max() < 2e-5


def test_unsmoothed_rigidness(vd, oracle_lib, scene):
    w = scene
    rng = np.random.default_rng(40)
    depth, rig = f32_state(rng, w)
    g = _gpu_window(vd, w)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), 256, depth, rig, w.poses)
    g.rigidness_update()
    _, _, W_gpu = g.get_pose_depth_rigidness(poses=False, depth=False)
    W_ref = ow.emissions()
    # per-pixel log-likelihood ell = log W: 1e-5 relative, plus the FP32
    # rounding of the stored W
    ell_ref = np.log(W_ref)
    err = np.abs(np.log(W_gpu.astype(np.float64)) - ell_ref)
    assert np.all(err <= 1e-5 * np.abs(ell_ref) + 2.0 ** -23), err.max()


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_depth_sweep(vd, oracle_lib, scene, k):
    w = scene
    rng = np.random.default_rng(50 + k)
    depth, rig = f32_state(rng, w)
    q = rng.uniform(0, 1, size=(w.T, w.H, w.W)).astype(np.float32)
    g = _gpu_window(vd, w)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=k)
    g.set_buffer(vd.BUF_SMOOTHED, q)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), 256, depth, rig, w.poses)
    g.depth_update(k)
    lab_gpu = g.get_buffer(vd.BUF_LABELS, (w.H, w.W), np.uint8)
    _, D_gpu, _ = g.get_pose_depth_rigidness(poses=False, rigidness=False)
    lab_ref = ow.mie_sweep(k, q.astype(np.float64))
    same = np.mean(lab_gpu == lab_ref)
    assert same >= 0.999, same
    agree = np.abs(D_gpu - ow.theta) <= 1e-5 * ow.theta
    assert np.mean(agree) >= 0.999
