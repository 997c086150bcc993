"""Batched windows (one CUDA graph for many windows of different sizes and T)
and the dense-scoring autotuner."""
import numpy as np
import pytest

from paper_2104_06789_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


def _windows():
    return [synthetic.small_planes(seed=4000, W=64, H=48, f=48.0, T=2),
            synthetic.small_planes(seed=4001, W=96, H=72, f=72.0, T=3),
            synthetic.handheld(seed=4002, W=80, H=60, f=66.0, T=4),
            synthetic.small_planes(seed=4003, W=128, H=96, f=96.0, T=3)]


def _make(vd, w, i):
    p = vd.default_params(hyps_per_frame=128, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1], window_id=i)
    g = vd.Window(w.flows.astype(np.float16), w.K, p)
    g.bootstrap(w.poses[0])
    return g


def test_batch_equals_individual_windows(vd):
    ws = _windows()
    solo = []
    for i, w in enumerate(ws):
        g = _make(vd, w, i)
        g.em_step(2)
        solo.append(g.get_pose_depth_rigidness())
        g.destroy()
    gs = [_make(vd, w, i) for i, w in enumerate(ws)]
    b = vd.Batch(gs, 2)
    lat = b.run()
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    for g, (P, D, Wm) in zip(gs, solo):
        P2, D2, W2 = g.get_pose_depth_rigidness()
        assert np.array_equal(P, P2) and np.array_equal(D, D2) and np.array_equal(Wm, W2)
    # a second run continues the iterations of every window, like em_step
    b.run()
    for i, (g, w) in enumerate(zip(gs, ws)):
        h = _make(vd, w, i)
        h.em_step(4)
        assert np.array_equal(h.get_pose_depth_rigidness()[0], g.get_pose_depth_rigidness()[0])
        h.destroy()
    b.destroy()
    for g in gs:
        g.destroy()


def test_batch_rejects_bad_input(vd):
    w = _windows()[0]
    g = _make(vd, w, 0)
    with pytest.raises(vd.VoldorError):
        vd.Batch([g, g], 1)
    p = vd.default_params(hyps_per_frame=64)
    raw = vd.Window(w.flows.astype(np.float32), w.K, p)           # not bootstrapped
    with pytest.raises(vd.VoldorError) as e:
        vd.Batch([g, raw], 1)
    assert e.value.status == vd.ERR_NOT_BOOTSTRAPPED
    g.destroy()
    raw.destroy()


def test_autotune_keeps_results(vd):
    w = synthetic.small_planes(seed=4010, W=160, H=120, f=120.0, T=3)
    a = _make(vd, w, 0)
    hpt, chunks, ms = a.autotune()
    assert hpt in (2, 4, 8) and chunks >= 1 and ms > 0
    a.em_step(2)
    b = _make(vd, w, 0)
    b.set_score_shape({2: 4, 4: 8, 8: 2}[hpt], 1)
    b.em_step(2)
    Pa, Da, _ = a.get_pose_depth_rigidness()
    Pb, Db, _ = b.get_pose_depth_rigidness()
    # another tile shape only reorders the FP64 sums of the dense scores
    assert np.abs(Pa - Pb).max() < 1e-9
    assert np.mean(Da == Db) > 0.999


def test_autotune_hyps_on_a_window(vd):
    """The hypothesis-count autotuner on the library's windows: an impossible
    tolerance keeps the window's own count, an unbounded one takes the
    smallest candidate, and the chosen count's window runs."""
    from paper_2104_06789_gb300 import synthetic, tuning
    w = synthetic.small_planes(seed=1003)
    p = vd.default_params(hyps_per_frame=256, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1])
    flows = w.flows.astype(np.float32)
    S, tried, _ = tuning.autotune_hyps(flows, w.K, p, w.poses[0], rot_tol=-1.0, trans_tol=-1.0)
    assert S == 256 and [s for s, _, _ in tried] == [64, 128]
    S, tried, _ = tuning.autotune_hyps(flows, w.K, p, w.poses[0], rot_tol=np.inf, trans_tol=np.inf)
    assert S == 64 and len(tried) == 1
    S, tried, (rt, tt) = tuning.autotune_hyps(flows, w.K, p, w.poses[0])
    assert S in (64, 128, 256) and np.isfinite(rt) and np.isfinite(tt)
    for s, ang, rel in tried:
        assert np.isfinite(ang) and np.isfinite(rel)
