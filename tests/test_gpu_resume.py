"""Checkpoint / resume and determinism of the whole loop on the GPU.

A window's state between iterations is (poses, depth, unsmoothed rigidness,
iteration counter k); the random draws are counter-based (Philox keyed by the
window, counters (index, t, k, stream)) and every reduction runs in a fixed
order. So a run stopped after some iterations, read out through the C ABI,
written into a fresh context with voldor_set_state and continued gives the
same result bit for bit as the run that never stopped, and two contexts built
from the same input agree bit for bit."""
import numpy as np
import pytest

from tests.helpers import small_window

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


def _window(vd, w, S=256):
    p = vd.default_params(hyps_per_frame=S, inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1])
    return vd.Window(w.flows.astype(np.float16), w.K, p)


def test_resume_from_a_saved_state_is_bit_exact(vd):
    w = small_window(seed=1000)
    a = _window(vd, w)
    a.bootstrap(w.poses[0])
    a.em_step(3)
    ref = a.get_pose_depth_rigidness()
    a.destroy()

    b = _window(vd, w)
    b.bootstrap(w.poses[0])
    b.em_step(1)
    P, D, Wm = b.get_pose_depth_rigidness()                # the checkpoint
    b.destroy()
    c = _window(vd, w)
    c.set_state(poses=P, depth=D, rigidness=Wm, iteration=1)
    c.em_step(2)
    got = c.get_pose_depth_rigidness()
    c.destroy()
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)


def test_two_contexts_agree_bit_for_bit(vd):
    w = small_window(seed=1001)
    out = []
    for _ in range(2):
        g = _window(vd, w)
        g.bootstrap(w.poses[0])
        g.em_step(2)
        out.append(g.get_pose_depth_rigidness())
        g.destroy()
    for x, y in zip(*out):
        assert np.array_equal(x, y)
