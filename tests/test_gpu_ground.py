"""Ground-plane scale through the C ABI against the oracle, teacher-forced on
the same FP32 depth and rigidness: the scale agrees to 1e-4 (the histogram
bins are decided in FP64 on both sides; a pixel whose height sits on a bin
edge can fall either way, moving the centroid by ~1e-6), applying it scales
the depth and every translation, and a scene without ground is degenerate."""
import numpy as np
import pytest

import oracle
from paper_2104_06789_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


def _state(w, s=1.0):
    lo, hi = 1.0 / w.inv_depth_range[1], 1.0 / w.inv_depth_range[0]
    depth = np.clip(np.nan_to_num(w.depth0, nan=hi) * s, lo, hi).astype(np.float32)
    rig = np.broadcast_to(w.rigid[0].astype(np.float32), (w.T,) + w.rigid.shape[1:]).copy()
    return depth, rig


@pytest.mark.parametrize("seed,s", [(3000, 1.0), (3001, 0.5)])
def test_scale_matches_the_oracle(vd, seed, s):
    w = synthetic.driving(seed=seed, W=414, H=125, f=239.3, T=2)
    depth, rig = _state(w, s)
    p = vd.default_params(inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1],
                          hyps_per_frame=64)
    g = vd.Window(w.flows.astype(np.float32), w.K, p)
    g.bootstrap(w.poses[0])
    g.set_state(poses=w.poses, depth=depth, rigidness=rig)
    sc = g.ground_scale(1.65)
    ow = oracle.OracleWindow(w.flows, w.K, inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1])
    ow.theta[:] = depth.astype(np.float64)
    ow.wmap[:] = rig.astype(np.float64)
    st, sc_or, mode, n = ow.ground_scale(1.65)
    assert st == 0 and n > 1000
    assert sc == pytest.approx(sc_or, rel=1e-4)
    assert sc == pytest.approx(1.0 / s, rel=2e-2)           # the scene's ground is 1.65 m below the camera
    # applying it
    P0, D0, _ = g.get_pose_depth_rigidness(rigidness=False)
    sc2 = g.ground_scale(1.65, apply=True)
    assert sc2 == sc
    P1, D1, _ = g.get_pose_depth_rigidness(rigidness=False)
    assert np.allclose(D1, (D0.astype(np.float64) * sc).astype(np.float32), rtol=1e-7)
    assert np.allclose(P1[:, :3, 3], P0[:, :3, 3] * sc, rtol=1e-12)
    assert np.array_equal(P1[:, :3, :3], P0[:, :3, :3])
    g.destroy()


def test_no_ground_is_degenerate(vd):
    w = synthetic.small_planes(seed=1000)
    p = vd.default_params(inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1],
                          hyps_per_frame=64)
    g = vd.Window(w.flows.astype(np.float32), w.K, p)
    assert vd.lib().voldor_ground_scale(g._h, 1.65, 0.17, 0, None) == vd.ERR_NOT_BOOTSTRAPPED
    g.bootstrap(w.poses[0])
    flat = np.full((w.H, w.W), 10.0, np.float32)           # a fronto-parallel wall: normals along z
    g.set_state(depth=flat)
    with pytest.raises(vd.VoldorError) as ei:
        g.ground_scale(1.65)
    assert ei.value.status == vd.ERR_DEGENERATE
    for h, tilt in [(0.0, 0.17), (-1.0, 0.17), (1.65, 0.0), (1.65, 1.6), (float("nan"), 0.17)]:
        assert vd.lib().voldor_ground_scale(g._h, h, tilt, 0, None) == vd.ERR_INVALID_ARG
    g.destroy()
