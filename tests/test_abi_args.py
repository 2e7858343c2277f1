"""CPU-side checks of csfmm_plan_create's argument validation: the checks that
come before any device pointer is inspected return CSFMM_ERR_INVALID_ARG with a
message naming the argument, and write no plan.  No GPU is needed."""
import ctypes

import pytest

from paper_2508_13550_gb300 import csfmm as C

INVALID_ARG = 1


@pytest.fixture(scope="module")
def lib():
    from paper_2508_13550_gb300 import build
    L = ctypes.CDLL(build.build())
    L.csfmm_plan_create.restype = ctypes.c_int
    L.csfmm_plan_create.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    L.csfmm_last_error.restype = ctypes.c_char_p
    return L


def _create(L, N=100, kernel=0, degree=8, theta=0.7, max_leaf=64, opt=None):
    out = ctypes.c_void_p(12345)
    rc = L.csfmm_plan_create(None, N, kernel, degree, theta, max_leaf,
                             ctypes.byref(opt) if opt is not None else None, None,
                             ctypes.byref(out))
    return rc, out.value, L.csfmm_last_error().decode()


@pytest.mark.parametrize("kw,word", [
    (dict(N=0), "N must be"),
    (dict(N=1 << 31), "N must be"),
    (dict(kernel=7), "kernel"),
    (dict(degree=0), "degree"),
    (dict(degree=17), "degree"),
    (dict(theta=0.0), "theta"),
    (dict(theta=1.0), "theta"),
    (dict(theta=float("nan")), "theta"),
    (dict(max_leaf=0), "max_leaf"),
])
def test_bad_arguments_are_refused(lib, kw, word):
    rc, out, msg = _create(lib, **kw)
    assert rc == INVALID_ARG and out is None and word in msg, (kw, rc, msg)


def test_bad_options_are_refused(lib):
    opt = C.Options(5, 16, 0, 0, 0, 0, 0)  # unknown precision
    rc, out, msg = _create(lib, opt=opt)
    assert rc == INVALID_ARG and out is None and "precision" in msg
    opt = C.Options(C.FP32_BULK, 65, 0, 0, 0, 0, 0)  # more right-hand sides than supported
    rc, out, msg = _create(lib, opt=opt)
    assert rc == INVALID_ARG and out is None and "max_nrhs" in msg


def test_null_output_handle_is_refused(lib):
    rc = lib.csfmm_plan_create(None, 100, 0, 8, 0.7, 64, None, None, None)
    assert rc == INVALID_ARG and "out" in lib.csfmm_last_error().decode()
