"""The expiry path of the bounded device-side waits, without a GPU fault: the
library's bounded mbarrier wait, run on a phase that nothing completes, gives
up after its poll limit and the call reports VOLDOR_ERR_TIMEOUT; the context
and the device stay usable (a window runs and matches a run made before)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


def _run_window(vd):
    from paper_2104_06789_gb300 import synthetic
    w = synthetic.small_planes(seed=1000)
    p = vd.default_params(hyps_per_frame=128, inv_depth_min=w.inv_depth_range[0],
                          inv_depth_max=w.inv_depth_range[1])
    g = vd.Window(w.flows.astype(np.float32), w.K, p)
    g.bootstrap(w.poses[0])
    g.em_step(2)
    out = g.get_pose_depth_rigidness()
    g.destroy()
    return out


def test_bounded_wait_expires_and_reports_timeout(vd):
    before = _run_window(vd)
    short_st, short_cyc = vd.probe_bounded_wait(1000)
    long_st, long_cyc = vd.probe_bounded_wait(100000)
    assert short_st == vd.ERR_TIMEOUT and long_st == vd.ERR_TIMEOUT
    assert 0 < short_cyc < long_cyc                 # the wait polled for its whole budget, then gave up
    assert vd.probe_bounded_wait(0)[0] == vd.ERR_TIMEOUT
    assert vd.lib().voldor_probe_bounded_wait(-1, None) == vd.ERR_INVALID_ARG
    after = _run_window(vd)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
