"""Edge cases of the pose update against the oracle: a frame with no pixel
that has a 3D-2D correspondence (no group can be drawn: the update is
degenerate on both sides and the pose is kept), and the largest hypothesis
count the library accepts (S = 65536, a budget of 4S = 262,144 groups): the
collection keeps exactly S hypotheses, the same groups, slots and weights as
the oracle, and sampled dense scores agree to 1e-5."""
import numpy as np
import pytest

from tests.helpers import f32_state, oracle_window, small_window

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


def test_frame_without_correspondences_is_degenerate(vd, oracle_lib):
    w = small_window(seed=1000)
    rng = np.random.default_rng(70)
    depth, rig = f32_state(rng, w)
    poses = w.poses.copy()
    poses[0][:3, 3] = [500.0, 0.0, 0.0]            # camera 1 far to the side: no pixel projects into I_1
    p = vd.default_params(hyps_per_frame=128, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1])
    g = vd.Window(w.flows.astype(np.float32), w.K, p)
    g.set_state(poses=poses, depth=depth, rigidness=rig, iteration=0)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), 128, depth, rig, poses)
    assert ow.valid_pixels(2).size == 0
    st = g.pose_update(0, 2)
    assert st == vd.ERR_DEGENERATE
    hg = g.hypotheses()
    assert len(hg["group"]) == 0
    R, tv, wts, grp, slot = ow.collect_hypotheses(0, 2)
    assert len(grp) == 0
    st_o, n, _, _, _ = ow.pose_update(0, 2)
    assert st_o != 0 and n == 0
    P, _, _ = g.get_pose_depth_rigidness(depth=False, rigidness=False)
    assert np.array_equal(P[1], poses[1])           # the frame keeps its pose
    g.destroy()


def test_largest_hypothesis_count(vd, oracle_lib):
    w = small_window(seed=1000)
    rng = np.random.default_rng(71)
    depth, rig = f32_state(rng, w)
    rig = (0.5 + 0.5 * rig).astype(np.float32)
    S = 65536
    p = vd.default_params(hyps_per_frame=S, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1])
    assert p.groups_per_frame == 4 * S
    g = vd.Window(w.flows.astype(np.float32), w.K, p)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=1)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), S, depth, rig, w.poses)
    t = 2
    g.pose_update(1, t)
    hg = g.hypotheses()
    R, tv, wts, grp, slot = ow.collect_hypotheses(1, t)
    assert len(R) == S and len(hg["R"]) == S
    assert np.array_equal(hg["group"], grp) and np.array_equal(hg["slot"], slot)
    assert np.array_equal(hg["weight"], wts)
    assert np.abs(hg["R"] - R).max() < 1e-9
    dt = np.linalg.norm(hg["t"] - tv, axis=1) / np.maximum(np.linalg.norm(tv, axis=1), 1.0)
    assert dt.max() < 1e-9
    # dense scores of the FP32 scoring form, sampled across the tiles (the last one included)
    f32 = g.get_buffer(vd.BUF_HYPS_F32, (S, 12), np.float32).astype(np.float64)
    idx = np.array([0, 1, 511, 512, 4095, 30000, 65535 - 512, 65535])
    Rf = np.eye(3) + f32[idx, :9].reshape(-1, 3, 3)
    L_ref = ow.score(t, Rf, f32[idx, 9:])
    rel = np.abs(hg["L"][idx] - L_ref) / np.abs(L_ref)
    assert rel.max() < 1e-5, rel.max()
    g.destroy()
