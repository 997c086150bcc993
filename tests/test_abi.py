"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function include/voldor.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


def declared_functions():
    src = open(os.path.join(ROOT, "include", "voldor.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(voldor_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(vd):
    lib = ctypes.CDLL(vd.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_default_params_are_the_papers(vd):
    p = vd.default_params()
    assert (p.a1, p.a2, p.b1, p.b2) == (0.01, 0.09, -0.0022, 1.0)
    assert (p.lambda_, p.gamma, p.sigma_t, p.sigma_r) == (0.15, 0.9, 0.1, 0.004)
    assert p.criterion == vd.CRITERION_MIE
    assert p.residual == vd.RESIDUAL_FISK


def test_invalid_arguments_are_rejected_on_the_host(vd):
    L = vd.lib()
    K = vd.Intrinsics(100.0, 100.0, 10.0, 10.0)
    h = ctypes.c_void_p()
    flows = np.zeros((2, 8, 8, 2), np.float32)
    p = vd.default_params()
    fp = ctypes.c_void_p(flows.ctypes.data)
    assert L.voldor_init_window(None, 8, 8, 2, ctypes.byref(K), ctypes.byref(p), fp, 0, 0, None) == vd.ERR_INVALID_ARG
    for (w, hgt, T) in [(1, 8, 2), (8, 1, 2), (8, 8, 0), (8, 8, 17), (4097, 8, 2), (8, 4097, 2)]:
        assert L.voldor_init_window(ctypes.byref(h), w, hgt, T, ctypes.byref(K), ctypes.byref(p), fp, 0, 0,
                                    None) == vd.ERR_INVALID_ARG
        assert not h.value
    bad = vd.Intrinsics(0.0, 100.0, 10.0, 10.0)
    assert L.voldor_init_window(ctypes.byref(h), 8, 8, 2, ctypes.byref(bad), ctypes.byref(p), fp, 0, 0,
                                None) == vd.ERR_INVALID_ARG
    assert L.voldor_init_window(ctypes.byref(h), 8, 8, 2, ctypes.byref(K), ctypes.byref(p), fp, 7, 0,
                                None) == vd.ERR_INVALID_ARG
    for field, val in [("gamma", 1.0), ("gamma", 0.0), ("hyps_per_frame", 0), ("sigma_t", -1.0),
                       ("inv_depth_max", 0.01), ("x_min", 0.0), ("ms_max_iter", 0), ("a1", float("nan")),
                       ("criterion", 2), ("criterion", -1), ("residual", 2), ("residual", -1)]:
        q = vd.default_params(**{field: val})
        assert L.voldor_init_window(ctypes.byref(h), 8, 8, 2, ctypes.byref(K), ctypes.byref(q), fp, 0, 0,
                                    None) == vd.ERR_INVALID_ARG, field
    # NULL contexts
    assert L.voldor_em_step(None, 1) == vd.ERR_INVALID_ARG
    assert L.voldor_bootstrap(None, 0, None) == vd.ERR_INVALID_ARG
    L.voldor_destroy(None)
    assert vd.status_string(vd.ERR_DEGENERATE)


def test_product_path_does_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_2104_06789_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "or_window" not in txt and "liboracle" not in txt, f


def test_net_arguments_are_checked_on_the_host(vd):
    from oracle import conv_net
    L = vd.lib()
    for T in (1, 2, 5, 8):
        assert L.voldor_net_num_params(T) == conv_net.num_params(T)
    assert L.voldor_net_num_params(0) == 0 and L.voldor_net_num_params(9) == 0
    h = ctypes.c_void_p()
    assert L.voldor_net_create(0, ctypes.byref(h)) == vd.ERR_INVALID_ARG
    assert L.voldor_net_create(9, ctypes.byref(h)) == vd.ERR_INVALID_ARG
    assert L.voldor_net_create(2, None) == vd.ERR_INVALID_ARG
    assert L.voldor_net_forward(None, None, 0, 1, 1, 1, None, None) == vd.ERR_INVALID_ARG
    assert L.voldor_bootstrap_learned(None, None, None, 3) == vd.ERR_INVALID_ARG
    assert L.voldor_bootstrap_epipolar(None, 64, 1.0, None) == vd.ERR_INVALID_ARG
    assert L.voldor_ground_scale(None, 1.65, 0.17, 0, None) == vd.ERR_INVALID_ARG
    L.voldor_net_destroy(None)


def test_binding_checks_the_shapes_the_c_calls_read(vd):
    """The C calls that take host arrays read a size implied by the window
    (T x 4 x 4 poses, H x W depth, n x 3 x 3 rotations ...): the binding
    rejects arrays of any other shape before the call."""
    import numpy as np
    vd._require_shape("T1", np.eye(4), (4, 4))
    for bad in (np.eye(3), np.zeros(16), np.zeros((2, 4, 4))):
        with pytest.raises(ValueError):
            vd._require_shape("T1", bad, (4, 4))


def test_header_is_plain_c():
    """include/voldor.h is consumable from C (C99) as well as C++."""
    import shutil
    import subprocess
    hdr = os.path.join(ROOT, "include", "voldor.h")
    for cc, args in (("gcc", ["-std=c99", "-x", "c"]), ("g++", ["-std=c++11", "-x", "c++"])):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not found")
        r = subprocess.run([cc, "-fsyntax-only", "-Wall", "-Werror", *args, hdr], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
