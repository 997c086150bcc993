"""Host logic of the hypothesis-count autotuner, with a stand-in window whose
poses approach the reference as S grows (no GPU)."""
import numpy as np
import pytest

from paper_2104_06789_gb300 import tuning, voldor


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


class FakeWindow:
    """Poses = truth perturbed by err0 * (S_max / S - 1) + spread * (seed - 7)
    (rotation in rad, translation relative)."""
    made = []

    def __init__(self, truth, S_max, err0, params, spread=0.0):
        self.truth, self.S_max, self.err0, self.p, self.spread = truth, S_max, err0, params, spread
        FakeWindow.made.append((params.hyps_per_frame, params.groups_per_frame, params.seed))

    def bootstrap(self, T1):
        self.booted = True

    def em_step(self, n):
        assert self.booted and n == 5

    def get_pose_depth_rigidness(self, depth=True, rigidness=True):
        e = self.err0 * (self.S_max / self.p.hyps_per_frame - 1.0) + self.spread * (self.p.seed - 7)
        P = self.truth.copy()
        for t in range(len(P)):
            P[t, :3, :3] = _rot([1, 2, 3], e) @ P[t, :3, :3]
            P[t, :3, 3] *= 1.0 + e
        return P, None, None

    def destroy(self):
        pass


def _truth(T=4):
    P = np.tile(np.eye(4), (T, 1, 1))
    P[:, :3, 3] = [0.1, 0.0, 1.0]
    return P


@pytest.mark.parametrize("err0,expect", [(1e-6, 512), (2e-4, 1024), (6e-4, 2048), (1e-2, 4096)])
def test_smallest_agreeing_count_is_chosen(err0, expect):
    truth = _truth()
    params = voldor.Params(hyps_per_frame=4096, groups_per_frame=16384, seed=7)
    FakeWindow.made = []
    mk = lambda f, K, p: FakeWindow(truth, 4096, err0, p)
    S, tried, tol = tuning.autotune_hyps(None, (1, 1, 0, 0), params, np.eye(4), make_window=mk, rot_tol=1e-3,
                                         trans_tol=1e-3)
    assert S == expect and tol == (1e-3, 1e-3)
    # the reference ran first, with the window's own counts and key; groups scale with S
    assert FakeWindow.made[0] == (4096, 16384, 7)
    assert all(g == 4 * h and sd == 7 for h, g, sd in FakeWindow.made)
    assert [s for s, _, _ in tried] == [512, 1024, 2048][:len(tried)]
    assert params.hyps_per_frame == 4096            # the caller's parameters are untouched


@pytest.mark.parametrize("err0,expect", [(1e-4, 512), (3e-4, 1024), (8e-4, 2048), (3e-3, 4096)])
def test_default_bound_is_the_reference_spread(err0, expect):
    """Without explicit bounds a second full-count run with the next Philox
    key sets them; a candidate is accepted when no farther from the reference
    than that run."""
    truth = _truth()
    params = voldor.Params(hyps_per_frame=4096, groups_per_frame=16384, seed=7)
    FakeWindow.made = []
    mk = lambda f, K, p: FakeWindow(truth, 4096, err0, p, spread=1e-3)
    S, tried, (rt, tt) = tuning.autotune_hyps(None, (1, 1, 0, 0), params, np.eye(4), make_window=mk)
    assert S == expect
    assert FakeWindow.made[1] == (4096, 16384, 8)                  # the spread run
    assert rt == pytest.approx(1e-3, rel=1e-6) and tt == pytest.approx(1e-3, rel=1e-6)


def test_candidates_and_agreement_measure():
    assert tuning.default_candidates(8192) == [1024, 2048, 4096]
    assert tuning.default_candidates(256) == [64, 128]
    P = _truth(2)
    Q = P.copy()
    Q[1, :3, :3] = _rot([0, 0, 1], 0.01) @ Q[1, :3, :3]
    Q[0, :3, 3] *= 1.02
    ang, rel = tuning.pose_agreement(Q, P)
    assert ang == pytest.approx(0.01, rel=1e-9)
    assert rel == pytest.approx(0.02, rel=1e-9)
    with pytest.raises(ValueError):
        tuning.autotune_hyps(None, (1, 1, 0, 0), voldor.Params(hyps_per_frame=64), np.eye(4), candidates=[128],
                             make_window=lambda f, K, p: None)
