"""Host-side checks of the C ABI library (no GPU needed): it builds for
sm_103a, loads, and exports every function include/rsfde.h declares; plus
the seeded workload generators."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2102_11576_gb300 import _build, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rsfde.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rsfde_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rsfde_setup", "rsfde_solve", "rsfde_step", "rsfde_adjoint",
                     "rsfde_set_params", "rsfde_destroy", "rsfde_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(libpath):
    lib = ctypes.CDLL(libpath)
    lib.rsfde_strerror.restype = ctypes.c_char_p
    assert lib.rsfde_strerror(-4) == b"GMRES did not converge within max_iter"
    assert lib.rsfde_strerror(0) == b"ok"
    # argument validation happens before any CUDA call
    lib.rsfde_setup.restype = ctypes.c_int
    out = ctypes.c_void_p()
    assert lib.rsfde_setup(ctypes.byref(out), None, None, ctypes.c_double(1.5),
                           ctypes.c_double(1.5), ctypes.c_double(1.0), ctypes.c_double(1.0),
                           ctypes.c_double(0.1), ctypes.c_double(1e-3), None) == -1
    assert lib.rsfde_kernel_launches(None) == 0
    # grid sides beyond 4096 (convolution length 16384) are rejected before any CUDA call
    from paper_2102_11576_gb300 import _Grid
    byte = ctypes.c_uint8(1)
    for n1, n2 in ((4097, 8), (8, 4097), (0, 8)):
        g = _Grid(n1, n2, -1.0, 1.0, -1.0, 1.0)
        assert lib.rsfde_setup(ctypes.byref(out), ctypes.byref(g), ctypes.byref(byte), ctypes.c_double(1.5),
                               ctypes.c_double(1.5), ctypes.c_double(1.0), ctypes.c_double(1.0),
                               ctypes.c_double(0.1), ctypes.c_double(1e-3), None) == -1


def test_workload_geometry():
    w = workloads.make("polygon2048", n=256)
    X, Y = workloads.grid_xy(256, 256)
    m = w["in_omega"].astype(bool)
    assert m.any() and (~m).any()
    assert np.all(X[m] ** 2 + Y[m] ** 2 <= 1.0 + 1e-12)  # inscribed in the unit circle
    # convex: the mask along any row is one contiguous run
    for row in m:
        idx = np.nonzero(row)[0]
        if idx.size:
            assert idx[-1] - idx[0] + 1 == idx.size
    w = workloads.make("ellipse512", n=128)
    X, Y = workloads.grid_xy(128, 128)
    inside = X ** 2 / 0.81 + Y ** 2 / 0.36 <= 1
    assert np.array_equal(w["in_omega"].astype(bool), inside)
    assert np.all(w["u0"][~inside] == 0)
    w1, w2 = workloads.make("polygon2048", seed=3, n=64), workloads.make("polygon2048", seed=3, n=64)
    assert np.array_equal(w1["in_omega"], w2["in_omega"])  # seeded
