"""The whole VOLDOR loop (Table 1) against the FP64 oracle, iteration by
iteration: the config-1 window (160x120, f = 120, T = 3, S = 256, 3 EM
iterations) through voldor_em_step, and four small windows of mixed size and
T through one batched graph (voldor_batch_*).

Before each iteration the oracle takes the GPU's state (FP32 depth and
rigidness, FP64 poses, all exactly representable), so that a near-tie in one
iteration cannot cascade into the next; both then run one full iteration
(pose updates of every frame, E-step smoothing, MIE sweep, rigidness update)
on their own. Bounds, per iteration:
  - every frame's pose: 1e-6 rad and 1e-6 relative translation;
  - sweep labels identical on >= 99.9 % of pixels, and the depths equal to
    1e-6 relative there (the sampled candidates are drawn in FP32 on the GPU);
  - the rigidness update: log W within 1e-5 |log W| + 2^-23 at every (t, j),
    against the oracle evaluated at the GPU's resulting depth and poses.
"""
import numpy as np
import pytest

from tests.helpers import pose_close, small_window

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


def _oracle_iteration(ow, k):
    """One oracle iteration in Table 1's order, returning the sweep labels."""
    for t in range(1, ow.T + 1):
        ow.pose_update(k, t)
    em = ow.emissions()
    q = ow.smooth(0 if k % 2 == 0 else 1, em)
    labels = ow.mie_sweep(k, q)
    ow.rigidness()
    return labels


def _sync(ow, P, D, Wm):
    ow.poses[:] = P
    ow.theta[:] = D.astype(np.float64)
    ow.wmap[:] = Wm.astype(np.float64)


def _check_iteration(vd, oracle_lib, g, ow, flows64, w, k, S):
    """Runs the oracle's iteration k from its (synchronised) state and checks
    the GPU's result of the same iteration; returns the GPU state."""
    lab_ref = _oracle_iteration(ow, k)
    P, D, Wm = g.get_pose_depth_rigidness()
    lab = g.get_buffer(vd.BUF_LABELS, (w.H, w.W), np.uint8)
    for t in range(w.T):
        ok, ang, dt = pose_close(P[t], ow.poses[t])
        assert ok, (k, t, ang, dt)
    same = lab == lab_ref
    assert same.mean() >= 0.999, (k, same.mean())
    close = np.abs(D.astype(np.float64) - ow.theta) <= 1e-6 * ow.theta
    assert close[same].mean() >= 0.999, (k, close[same].mean())
    # the rigidness update at the GPU's own depth and poses
    ref = oracle_lib.OracleWindow(flows64, w.K, S=S, inv_depth_min=w.inv_depth_range[0],
                                  inv_depth_max=w.inv_depth_range[1])
    _sync(ref, P, D, Wm)
    ell_ref = np.log(ref.emissions())
    err = np.abs(np.log(Wm.astype(np.float64)) - ell_ref)
    assert np.all(err <= 1e-5 * np.abs(ell_ref) + 2.0 ** -23), (k, err.max())
    return P, D, Wm


def test_full_loop_config1_per_iteration(vd, oracle_lib):
    w = small_window(seed=1000)                        # 160x120, f = 120, T = 3
    S = 256
    flows32 = w.flows.astype(np.float32)
    flows64 = flows32.astype(np.float64)
    p = vd.default_params(hyps_per_frame=S, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1])
    g = vd.Window(flows32, w.K, p)
    g.bootstrap(w.poses[0])
    ow = oracle_lib.OracleWindow(flows64, w.K, S=S, inv_depth_min=w.inv_depth_range[0],
                                 inv_depth_max=w.inv_depth_range[1])
    ow.bootstrap(w.poses[0])
    P, D, Wm = g.get_pose_depth_rigidness()
    assert np.max(np.abs(D - ow.theta) / ow.theta) < 1e-6
    for k in range(3):
        _sync(ow, P, D, Wm)
        g.em_step(1)
        P, D, Wm = _check_iteration(vd, oracle_lib, g, ow, flows64, w, k, S)
    hyps = g.hypotheses()
    assert len(hyps["group"]) == S                     # the last frame kept exactly S
    g.destroy()


def test_batch_matches_the_oracle(vd, oracle_lib):
    """Four windows of mixed size and T in one graph (one iteration per run),
    each checked against its own oracle iteration by iteration."""
    shapes = [(160, 120, 3), (96, 72, 2), (128, 96, 4), (64, 48, 3)]
    S = 128
    wins, refs = [], []
    for i, (W, H, T) in enumerate(shapes):
        w = small_window(seed=1200 + i, W=W, H=H, f=0.75 * W, T=T)
        flows32 = w.flows.astype(np.float32)
        flows64 = flows32.astype(np.float64)
        p = vd.default_params(hyps_per_frame=S, inv_depth_min=w.inv_depth_range[0],
                              inv_depth_max=w.inv_depth_range[1], window_id=i)
        g = vd.Window(flows32, w.K, p)
        g.bootstrap(w.poses[0])
        ow = oracle_lib.OracleWindow(flows64, w.K, S=S, inv_depth_min=w.inv_depth_range[0],
                                     inv_depth_max=w.inv_depth_range[1], window_id=i)
        wins.append((g, w, flows64))
        refs.append(ow)
    batch = vd.Batch([g for g, _, _ in wins], 1)
    state = [g.get_pose_depth_rigidness() for g, _, _ in wins]
    for k in range(2):
        for ow, st in zip(refs, state):
            _sync(ow, *st)
        batch.run()
        state = [_check_iteration(vd, oracle_lib, g, ow, flows64, w, k, S)
                 for (g, w, flows64), ow in zip(wins, refs)]
    batch.destroy()
    for g, _, _ in wins:
        g.destroy()


class _Lockstep:
    """A window for the sliding-window driver that runs the GPU window and an
    oracle window side by side: each bootstrap gives both the same T_1, and
    each EM iteration starts the oracle from the GPU's state; the largest pose
    differences are recorded and the oracle's poses of every window kept."""

    def __init__(self, vd, oracle_lib, flows, K, params, w):
        self.vd, self.lib, self.K, self.p, self.w = vd, oracle_lib, K, params, w
        self.g = vd.Window(flows, K, params)
        self.flows64 = np.asarray(flows, dtype=np.float32).astype(np.float64)
        self.oracle_poses, self.worst = [], (0.0, 0.0)

    def set_flows(self, flows):
        self.g.set_flows(flows)
        self.flows64 = np.asarray(flows, dtype=np.float32).astype(np.float64)

    def bootstrap(self, T1):
        self.g.bootstrap(T1)
        self.o = self.lib.OracleWindow(self.flows64, self.K, S=self.p.hyps_per_frame,
                                       inv_depth_min=self.p.inv_depth_min, inv_depth_max=self.p.inv_depth_max)
        self.o.bootstrap(T1)
        _, D, _ = self.g.get_pose_depth_rigidness(poses=False, rigidness=False)
        assert np.max(np.abs(D - self.o.theta) / self.o.theta) < 1e-6
        self.k = 0

    def em_step(self, n):
        for _ in range(n):
            _sync(self.o, *self.g.get_pose_depth_rigidness())
            self.g.em_step(1)
            _oracle_iteration(self.o, self.k)
            P, _, _ = self.g.get_pose_depth_rigidness(depth=False, rigidness=False)
            for t in range(P.shape[0]):
                ok, ang, dt = pose_close(P[t], self.o.poses[t])
                self.worst = (max(self.worst[0], ang), max(self.worst[1], dt))
            self.k += 1
        self.oracle_poses.append(self.o.poses.copy())

    def get_pose_depth_rigidness(self, **kw):
        return self.g.get_pose_depth_rigidness(**kw)

    def destroy(self):
        self.g.destroy()


class _Replay:
    """Hands the driver recorded per-window poses (the oracle's)."""

    def __init__(self, poses):
        self.poses = iter(poses)

    def set_flows(self, flows):
        pass

    def bootstrap(self, T1):
        pass

    def em_step(self, n):
        self.P = next(self.poses)

    def get_pose_depth_rigidness(self, **kw):
        return self.P, None, None


def test_sliding_window_vo_against_the_oracle(vd, oracle_lib):
    """A noisy driving-like sequence (207x63, 8 flows) through the sliding-window
    driver (windows of 4 flows, stride 2, 2 iterations), each window's T_1 the
    previous window's estimate: at every iteration of every window the GPU's
    poses agree with the oracle's (1e-6 rad, 1e-6 relative translation), and
    the trajectory the driver chains from the oracle's windows agrees with the
    GPU's: every relative pose to the same bound, and the chained camera
    centres to (frames) x 1e-6 of the path (each relative pose's error adds at
    most its own bound along the chain)."""
    from paper_2104_06789_gb300 import synthetic, vo
    w = synthetic.driving(seed=3002, W=207, H=63, f=119.7, T=8)
    p = vd.default_params(hyps_per_frame=256, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1])
    flows = w.flows.astype(np.float16).astype(np.float32)
    holder = {}

    def make(f, K, params):
        holder["win"] = _Lockstep(vd, oracle_lib, f, K, params, w)
        return holder["win"]

    drv = vo.SlidingWindowVO(w.K, T=4, stride=2, n_iters=2, params=p, make_window=make)
    r = drv.run(flows, T1=w.poses[0])
    lock = holder["win"]
    assert r["starts"] == [0, 2, 4]
    assert lock.worst[0] <= 1e-6 and lock.worst[1] <= 1e-6, lock.worst
    ro = vo.SlidingWindowVO(w.K, T=4, stride=2, n_iters=2,
                            make_window=lambda f, K, params: _Replay(lock.oracle_poses)).run(flows, T1=w.poses[0])
    for a, b in zip(r["relative"], ro["relative"]):
        ok, ang, dt = pose_close(a, b)
        assert ok, (ang, dt)
    c = np.array([-M[:3, :3].T @ M[:3, 3] for M in r["trajectory"]])
    co = np.array([-M[:3, :3].T @ M[:3, 3] for M in ro["trajectory"]])
    path = np.linalg.norm(np.diff(c, axis=0), axis=1).sum()
    assert np.abs(c - co).max() <= len(c) * 1e-6 * path
