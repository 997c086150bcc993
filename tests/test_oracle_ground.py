"""Pins of the oracle's ground-plane scale: an exact ground plane, exact
equivariance under a depth scale of 2, the tilt threshold, and the driving
scene's ground at 1.65 m."""
import numpy as np
import pytest

import oracle
from paper_2104_06789_gb300 import synthetic


def _plane_window(h=1.65, W=160, H=120, f=120.0, pitch_deg=0.0):
    """Depth of a ground plane h below a camera pitched by pitch_deg (closed
    form per ray: the plane n . X = -h ... solved for the z-depth)."""
    cx, cy = (W - 1) / 2, (H - 1) / 2
    ys, xs = np.mgrid[0:H, 0:W].astype(float)
    d = np.stack([(xs - cx) / f, (ys - cy) / f, np.ones_like(xs)], -1)
    a = np.deg2rad(pitch_deg)
    n_up = np.array([0.0, np.cos(a), np.sin(a)])          # the ground's normal, pointing down from the camera
    dot = d @ n_up
    depth = np.where(dot > 1e-3, h / np.maximum(dot, 1e-3), 60.0)     # z-depth of the hit; sky far away
    flows = np.zeros((2, H, W, 2))
    ow = oracle.OracleWindow(flows, (f, f, cx, cy), inv_depth_min=1 / 100.0, inv_depth_max=1 / 0.1)
    ow.theta[:] = depth
    ow.wmap[:] = 1.0
    return ow


def test_exact_ground_plane_gives_the_height():
    ow = _plane_window(h=1.65)
    st, scale, mode, n = ow.ground_scale(1.65)
    assert st == 0 and n > 5000
    assert scale == pytest.approx(1.0, abs=2e-3)          # one histogram bin is 0.27 %
    assert 2 ** mode == pytest.approx(1.65, rel=2e-3)


def test_depth_scale_two_shifts_the_mode_exactly():
    ow = _plane_window(h=1.3)
    st, s1, m1, n1 = ow.ground_scale(1.3)
    ow.theta[:] *= 2.0
    ow.params.inv_depth_min /= 2.0                        # keep the range ends away from the doubled depths
    ow.params.inv_depth_max /= 2.0
    st2, s2, m2, n2 = ow.ground_scale(1.3)
    assert st2 == 0 and n2 == n1
    assert m2 == m1 + 1.0
    assert s2 == s1 / 2.0


def test_tilt_threshold():
    ow = _plane_window(h=1.65, pitch_deg=25.0)             # the ground normal is 25 deg off the camera's y axis
    st, scale, mode, n = ow.ground_scale(1.65, max_tilt_deg=10.0)
    assert n == 0 and st != 0
    st, scale, mode, n = ow.ground_scale(1.65, max_tilt_deg=30.0)
    assert st == 0 and scale == pytest.approx(1.0, abs=2e-3)


@pytest.mark.parametrize("seed", [3000, 3001])
def test_driving_scene_ground_height(seed):
    w = synthetic.driving(seed=seed, W=414, H=125, f=239.3, T=2, noise=False)
    ow = oracle.OracleWindow(w.flows, w.K, inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1])
    ow.theta[:] = np.nan_to_num(w.depth0, nan=1.0)
    ow.wmap[:] = w.rigid.astype(float)
    st, scale, mode, n = ow.ground_scale(1.65)
    assert st == 0 and scale == pytest.approx(1.0, rel=1e-2)
