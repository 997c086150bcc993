import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


def fronto_parallel_window(W=24, H=18, T=3, depth=5.0, f=30.0, shifts=None):
    """A fronto-parallel plane seen by a camera translating parallel to it:
    every flow field is constant, so bilinear sampling is exact and the true
    depth and poses are a noiseless fixed point of the model."""
    if shifts is None:
        shifts = [(0.05, -0.03), (0.04, 0.02), (-0.03, 0.05), (0.02, 0.04)][:T]
    K = (f, f, (W - 1) / 2.0, (H - 1) / 2.0)
    flows = np.zeros((T, H, W, 2))
    poses = np.tile(np.eye(4), (T, 1, 1))
    for t, (tx, ty) in enumerate(shifts):
        poses[t, 0, 3] = tx
        poses[t, 1, 3] = ty
        flows[t, ..., 0] = f * tx / depth
        flows[t, ..., 1] = f * ty / depth
    return flows, K, poses, np.full((H, W), depth)
