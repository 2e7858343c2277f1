"""The allocation-free evaluation entry point, csfmm_evaluate_static.

It serves callers that must not call cudaMalloc while they evaluate (a
serving loop whose free device memory is all promised to admitted requests,
or a host application that owns device memory through its own allocator).
Its scratch is one static device array shared by every call, so this test
checks, through the C ABI, that two calls in a row give the same potentials
as csfmm_evaluate bit for bit (the same kernels on the same data; the second
call must not see the first call's data), that the FP32-bulk form with one
right-hand side runs the mirrored-pair pass there too (same launch count),
and that a request larger than the array is refused with a clear message.

This file is collected last so that a failure here cannot hide another test.
"""
import ctypes

import numpy as np
import pytest

from paper_2508_13550_gb300 import inputs as I
from gpu_util import cuda_or_skip, dev

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 parity tolerance of the other GPU tests (here: bitwise)


@pytest.fixture(scope="module")
def env():
    torch = cuda_or_skip()
    from paper_2508_13550_gb300 import csfmm
    return torch, csfmm


def _call(C, fn, plan, w, out, stream):
    return getattr(C.load(), fn)(plan.handle, ctypes.c_void_p(w.data_ptr()), w.shape[0],
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("kernel,precision,nrhs",
                         [(0, 0, 1), (1, 1, 3), (2, 0, 5), (2, 1, 1), (0, 1, 1), (0, 1, 16)],
                         ids=["laplace-fp64", "biot-savart-fp32", "newton-fp64-5rhs",
                              "newton-fp32-1rhs", "laplace-fp32-1rhs", "laplace-fp32-16rhs"])
def test_static_scratch_matches_evaluate_twice(env, kernel, precision, nrhs):
    torch, C = env
    pts, A = I.cubed_sphere_grid(32)
    plan = C.plan_create(dev(torch, pts), kernel, 8, 0.7, 64, precision=precision,
                         max_nrhs=max(16, nrhs))
    if precision == 1 and nrhs == 1 and kernel != 1:
        assert C.plan_stats(plan)["sym_pairs"] > 0  # the mirrored-pair pass has work
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(kernel + 10 * precision)
    dim = C.kernel_dim(kernel)
    for call in range(2):  # a second call with other weights: no stale scratch
        w = dev(torch, rng.standard_normal((nrhs, len(pts))) * A)
        ref = torch.empty((nrhs, len(pts), dim), dtype=torch.float64, device="cuda")
        got = torch.full_like(ref, float("nan"))
        assert _call(C, "csfmm_evaluate", plan, w, ref, stream) == 0, C.last_error()
        launches = C.plan_stats(plan)["launches_per_evaluate"]
        assert _call(C, "csfmm_evaluate_static", plan, w, got, stream) == 0, C.last_error()
        assert C.plan_stats(plan)["launches_per_evaluate"] == launches
        torch.cuda.synchronize()
        C.plan_sync(plan)
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(g).all()
        assert _rel(g, r) <= TOL, (call, _rel(g, r))
        assert np.array_equal(g, r), call
    C.plan_destroy(plan)


def test_static_scratch_refuses_oversized_requests(env):
    torch, C = env
    pts, A = I.cubed_sphere_grid(128)  # 98,304 points
    plan = C.plan_create(dev(torch, pts), 0, 6, 0.7, 144)
    stream = torch.cuda.current_stream().cuda_stream
    nrhs = 64  # 64 x 98,304 x 8 bytes of weights alone exceed the 64 MiB array
    w = torch.zeros((nrhs, len(pts)), dtype=torch.float64, device="cuda")
    out = torch.zeros((nrhs, len(pts), 1), dtype=torch.float64, device="cuda")
    rc = _call(C, "csfmm_evaluate_static", plan, w, out, stream)
    assert rc == 1
    msg = C.last_error()
    assert "static scratch holds" in msg and str(C.STATIC_SCRATCH_BYTES) in msg
    # a request that fits still works after the refusal
    w1 = dev(torch, (I.real_sph_harm(4, 3, pts) * A)[None])
    ref = C.evaluate(plan, w1)
    got = C.evaluate_static(plan, w1)
    torch.cuda.synchronize()
    assert _rel(got.cpu().numpy(), ref.cpu().numpy()) <= TOL
    C.plan_destroy(plan)
