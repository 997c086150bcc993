"""Windows of extreme shape against the FP64 oracle: the smallest window the
library accepts (2x2), ragged ones (3x2, 7x5), strips one chain long and two
chains wide (1000x2 and 2x600: 2-pixel chains in the other direction), the
longest chain the depth sweep resolves in shared memory (4096x2) and the
largest T (16) on a small image.

Per shape, teacher-forced as in the stage parity tests (both sides get the
same FP32-representable state): the smoothed rigidness along rows and along
columns (Eqs. 11-14), the MIE sweep in all four directions (Eq. 10, Fig. 5:
labels and depths equal to the oracle's at every pixel outside the runs that
follow a near tie, see helpers.tie_runs; on the strips the depth varies so slowly
along a chain that candidates often score within 1e-7 of each other, below
what FP32 candidate scores can order),
the unsmoothed rigidness (Table 1) and the dense scores of a few hypotheses
(Eq. 10 on the pose), with the bounds of those tests. Then the whole loop
(bootstrap and two EM iterations) runs on the same window: every call
returns OK, or DEGENERATE where a frame yields no hypothesis (the 2x600
strip's second frame has no correspondence at all, which must give
DEGENERATE, as it does in the oracle), and every output
is finite and in range. Pose parity of the whole loop is not asserted here:
on a strip of pixels the rays of a minimal group are nearly coplanar, where
P3P is ill-conditioned and two correct solvers need not agree to 1e-9."""
import numpy as np
import pytest

from tests.helpers import f32_hypotheses, f32_state, oracle_window, small_window, tie_runs

pytestmark = pytest.mark.gpu

# (W, H, T)
SHAPES = [(2, 2, 1), (3, 2, 2), (7, 5, 2), (1000, 2, 2), (2, 600, 2), (4096, 2, 1), (24, 16, 16)]
S = 64


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


def _window(shape):
    W, H, T = shape
    return small_window(seed=1200 + W + H, W=W, H=H, f=max(W, H) * 0.75, T=T)


def _pair(vd, oracle_lib, w, rng, k):
    depth, rig = f32_state(rng, w)
    p = vd.default_params(hyps_per_frame=S, inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1])
    g = vd.Window(w.flows.astype(np.float32), w.K, p)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=k)
    ow = oracle_window(oracle_lib, w, w.flows.astype(np.float32).astype(np.float64), S, depth, rig, w.poses)
    return g, ow


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_stages_on_extreme_shapes(vd, oracle_lib, shape):
    w = _window(shape)
    rng = np.random.default_rng(shape[0] * 7 + shape[1])
    for k in (0, 1):                                   # smoothing along rows, then columns
        g, ow = _pair(vd, oracle_lib, w, rng, k)
        g.rigidness_smooth(k)
        q_gpu = g.get_buffer(vd.BUF_SMOOTHED, (w.T, w.H, w.W), np.float32)
        q_ref = ow.smooth(k % 2, ow.emissions())
        assert np.abs(q_gpu - q_ref).max() < 2e-5, (k, np.abs(q_gpu - q_ref).max())
        g.destroy()
    for k in range(4):                                 # L->R, T->B, R->L, B->T
        g, ow = _pair(vd, oracle_lib, w, rng, k)
        q = rng.uniform(0, 1, size=(w.T, w.H, w.W)).astype(np.float32)
        g.set_buffer(vd.BUF_SMOOTHED, q)
        g.depth_update(k)
        lab_gpu = g.get_buffer(vd.BUF_LABELS, (w.H, w.W), np.uint8)
        _, D_gpu, _ = g.get_pose_depth_rigidness(poses=False, rigidness=False)
        th0 = ow.theta.copy()
        lab_ref = ow.mie_sweep(k, q.astype(np.float64))
        tied = tie_runs(ow, k, q.astype(np.float64), th0, lab_ref, lab_gpu)
        assert tied.mean() <= 0.25, (k, tied.mean())   # most pixels are held to exact agreement
        same = lab_gpu == lab_ref
        assert np.all(same[~tied]), (k, np.argwhere(~same & ~tied)[:5])
        agree = np.abs(D_gpu - ow.theta) <= 1e-5 * ow.theta
        assert np.all(agree[~tied]), (k, np.argwhere(~agree & ~tied)[:5])
        g.destroy()
    g, ow = _pair(vd, oracle_lib, w, rng, 0)
    g.rigidness_update()
    _, _, W_gpu = g.get_pose_depth_rigidness(poses=False, depth=False)
    ell_ref = np.log(ow.emissions())
    err = np.abs(np.log(W_gpu.astype(np.float64)) - ell_ref)
    assert np.all(err <= 1e-5 * np.abs(ell_ref) + 2.0 ** -23), err.max()
    g.destroy()
    g, ow = _pair(vd, oracle_lib, w, rng, 0)           # scores weigh by the teacher-forced W
    R, tv = f32_hypotheses(rng, w.poses[0][:3, :3], w.poses[0][:3, 3], 5)
    L_gpu = g.score_hypotheses(1, R, tv)
    L_ref = ow.score(1, R, tv)
    assert np.all(L_ref < 0)
    rel = np.abs(L_gpu - L_ref) / np.abs(L_ref)
    assert rel.max() < 1e-5, rel.max()
    g.destroy()


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_whole_loop_runs_on_extreme_shapes(vd, oracle_lib, shape):
    w = _window(shape)
    p = vd.default_params(hyps_per_frame=S, inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1])
    g = vd.Window(w.flows.astype(np.float32), w.K, p)
    g.bootstrap(w.poses[0])
    ow = oracle_lib.OracleWindow(w.flows.astype(np.float32).astype(np.float64), w.K, S=S,
                                 inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1])
    ow.bootstrap(w.poses[0])
    _, D0, _ = g.get_pose_depth_rigidness(poses=False, rigidness=False)
    assert np.max(np.abs(D0 - ow.theta) / ow.theta) < 1e-6
    # a frame without a 3D-2D correspondence at the bootstrap state (in the
    # oracle) can draw no minimal group: its first pose update is degenerate
    no_corr = any(ow.valid_pixels(t).size == 0 for t in range(2, w.T + 1))
    st = [g.em_step(1) for _ in range(2)]
    assert all(s in (vd.OK, vd.ERR_DEGENERATE) for s in st), st
    if no_corr:
        assert st[0] == vd.ERR_DEGENERATE
    P, D, Wm = g.get_pose_depth_rigidness()
    assert np.all(np.isfinite(P)) and np.all(np.isfinite(D)) and np.all(np.isfinite(Wm))
    lo, hi = 1.0 / w.inv_depth_range[1], 1.0 / w.inv_depth_range[0]
    assert np.all(D >= lo * (1 - 1e-6)) and np.all(D <= hi * (1 + 1e-6))
    assert np.all(Wm >= 0) and np.all(Wm <= 1)
    for t in range(w.T):
        R = P[t, :3, :3]
        assert np.abs(R @ R.T - np.eye(3)).max() < 1e-9
    g.destroy()
