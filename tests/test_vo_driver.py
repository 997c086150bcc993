"""Host logic of the sliding-window driver (no GPU): window placement, pose
chaining, and how each window's T_1 and the kept poses come from the
windows before it, with a stand-in window that returns the true relative
poses at the scale of its T_1."""
import numpy as np
import pytest

from paper_2104_06789_gb300 import vo


def _rot(ax, ang):
    ax = np.asarray(ax, float) / np.linalg.norm(ax)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def _truth(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        T = np.eye(4)
        T[:3, :3] = _rot(rng.normal(size=3), rng.uniform(0, 0.05))
        T[:3, 3] = rng.normal(size=3) * 0.1
        out.append(T)
    return np.array(out)


class FakeWindow:
    """Frame indices travel in flows[:, 0, 0, 0]; the estimate of each
    relative pose is the truth with its translation scaled by the ratio of
    the bootstrap T_1's translation to the true one."""
    log = []

    def __init__(self, truth, flows):
        self.truth = truth
        self.set_flows(flows)

    def set_flows(self, flows):
        self.frames = [int(v) for v in flows[:, 0, 0, 0]]

    def bootstrap(self, T1):
        f = self.frames[0]
        self.scale = np.linalg.norm(T1[:3, 3]) / np.linalg.norm(self.truth[f][:3, 3])
        FakeWindow.log.append(("bootstrap", f, np.array(T1)))

    def bootstrap_epipolar(self, n, baseline):
        T1 = self.truth[self.frames[0]].copy()
        T1[:3, 3] *= baseline / np.linalg.norm(T1[:3, 3])
        self.bootstrap(T1)
        return T1

    def em_step(self, n):
        pass

    def ground_scale(self, h, tilt, apply=False):
        s = 1.0 / self.scale                 # the ground puts the window back at the true scale
        if apply:
            self.scale = 1.0
        return s

    def get_pose_depth_rigidness(self, **kw):
        P = np.array([self.truth[f].copy() for f in self.frames])
        P[:, :3, 3] *= self.scale
        return P, None, None


def _flows(n):
    f = np.zeros((n, 2, 2, 2), np.float32)
    f[:, 0, 0, 0] = np.arange(n)
    return f


@pytest.mark.parametrize("n,T,stride,expect", [(10, 4, 2, [0, 2, 4, 6]), (11, 4, 3, [0, 3, 6, 7]),
                                               (6, 6, 1, [0]), (7, 3, 1, [0, 1, 2, 3, 4])])
def test_window_starts(n, T, stride, expect):
    assert vo.window_starts(n, T, stride) == expect


def test_window_starts_rejects_non_overlapping():
    with pytest.raises(ValueError):
        vo.window_starts(10, 4, 4)
    with pytest.raises(ValueError):
        vo.window_starts(3, 4, 1)


def test_chain_composes_world_to_camera():
    truth = _truth(5)
    M = vo.chain(truth)
    assert np.allclose(M[0], np.eye(4))
    for f in range(1, 6):
        ref = np.eye(4)
        for T in truth[:f]:
            ref = T @ ref
        assert np.allclose(M[f], ref)


@pytest.mark.parametrize("n,T,stride", [(10, 4, 2), (11, 4, 3), (9, 6, 1)])
def test_driver_propagates_T1_and_keeps_each_pose_once(n, T, stride):
    truth = _truth(n, seed=n)
    FakeWindow.log = []
    d = vo.SlidingWindowVO((100.0, 100.0, 10.0, 10.0), T=T, stride=stride, n_iters=1,
                           make_window=lambda f, K, p: FakeWindow(truth, f))
    first = truth[0].copy()
    first[:3, 3] *= 2.0                                   # the caller's scale: twice the truth
    r = d.run(_flows(n), T1=first)
    scaled = truth.copy()
    scaled[:, :3, 3] *= 2.0                               # the scale travels through every window
    assert np.allclose(r["relative"], scaled)
    assert np.allclose(r["trajectory"], vo.chain(scaled))
    starts = vo.window_starts(n, T, stride)
    boots = [e for e in FakeWindow.log if e[0] == "bootstrap"]
    assert [b[1] for b in boots] == starts
    for b in boots[1:]:                                   # each window starts from the previous estimate
        assert np.allclose(b[2], scaled[b[1]])


def test_driver_epipolar_start_uses_the_baseline():
    truth = _truth(8, seed=3)
    d = vo.SlidingWindowVO((100.0, 100.0, 10.0, 10.0), T=4, stride=2, n_iters=1,
                           make_window=lambda f, K, p: FakeWindow(truth, f))
    r = d.run(_flows(8), T1=None, baseline=0.5)
    ratio = np.linalg.norm(r["relative"][:, :3, 3], axis=1) / np.linalg.norm(truth[:, :3, 3], axis=1)
    s = 0.5 / np.linalg.norm(truth[0][:3, 3])
    assert np.allclose(ratio, s)


def test_driver_ground_scale_restores_the_true_scale():
    truth = _truth(9, seed=5)
    d = vo.SlidingWindowVO((100.0, 100.0, 10.0, 10.0), T=4, stride=2, n_iters=1,
                           make_window=lambda f, K, p: FakeWindow(truth, f))
    first = truth[0].copy()
    first[:3, 3] *= 3.0
    r = d.run(_flows(9), T1=first, camera_height=1.65)
    assert np.allclose(r["relative"], truth)
