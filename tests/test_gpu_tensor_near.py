"""Near field of 16 right-hand sides on the tensor cores
(CSFMM_SCHED_TENSOR_NEAR): the kernel matrix formed on the fly as in the FP32
kernels, its products with the weights in TF32 with three products per term.
Compared with the oracle FMM on the same tree, degree and MAC (only the
GPU's rounding remains) within the per-case FP32 bar, and with the FP32-pipe
form of the same plan."""
import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I
from gpu_util import cuda_or_skip, dev
from fp32_bars import check as check32

pytestmark = pytest.mark.gpu

TENSOR_NEAR = 64


def _rel(a, b):
    return max(float(np.linalg.norm(a[r] - b[r]) / np.linalg.norm(b[r])) for r in range(len(b)))


def _eval(torch, C, pts, kernel, W, n, N0, schedule):
    P = C.plan_create(dev(torch, pts), kernel, n, 0.7, N0, precision=C.FP32_BULK, max_nrhs=16,
                      no_persistent=bool(schedule), schedule=schedule)
    out = C.evaluate(P, dev(torch, W)).cpu().numpy()[:, :, 0]
    C.plan_sync(P)
    return out


# degree 8 (P = 81: PC sources padded from 81 to 88) and 12 (P = 169)
CASES = [(O.KERNEL_LAPLACE, 8), (O.KERNEL_NEWTON, 12), (O.KERNEL_SAL, 8),
         (O.KERNEL_BIHARMONIC, 8), (O.KERNEL_ONE, 8)]


@pytest.mark.parametrize("kernel,n", CASES)
def test_tensor_near_matches_the_oracle(kernel, n):
    torch = cuda_or_skip()
    from paper_2508_13550_gb300 import csfmm as C
    pts, A = I.cubed_sphere_grid(48)
    coeffs = I.random_sh_coeffs(8, 16, seed=70 + kernel)
    F = I.sph_harm_combination(pts, coeffs, nrhs=16)
    if kernel == O.KERNEL_ONE:
        F = F + 2.0 * np.abs(F).max(axis=1, keepdims=True)  # K = 1: keep the sums away from 0
    W = F * A[None, :]
    N0 = 4 * n * n
    ref = O.FMM(pts, n, 0.7, N0).evaluate(kernel, W)[:, :, 0]
    tc = _eval(torch, C, pts, kernel, W, n, N0, TENSOR_NEAR)
    fp = _eval(torch, C, pts, kernel, W, n, N0, 0)
    check32(f"fmm32-tc-k{kernel}-n{n}-r16", _rel(tc, ref))
    check32(f"fmm32-tc-vs-fp32-k{kernel}-n{n}-r16", _rel(tc, fp))


def test_tensor_near_ragged_leaves():
    """Random points with a dense cap and leaves of up to 300 points: target
    passes beyond the first 256 rows, partly filled row tiles and source tiles
    that are not a multiple of 8."""
    torch = cuda_or_skip()
    from paper_2508_13550_gb300 import csfmm as C
    rng = np.random.default_rng(71)
    a = I.random_sphere_points(9000, 72)
    cap = a[a[:, 2] > 0.85]
    pts = np.concatenate([a, cap + 1e-3 * rng.standard_normal(cap.shape)])
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    W = rng.uniform(0.0, 1.0, (16, len(pts))) / len(pts)
    ref = O.FMM(pts, 6, 0.7, 300).evaluate(O.KERNEL_NEWTON, W)[:, :, 0]
    tc = _eval(torch, C, pts, O.KERNEL_NEWTON, W, 6, 300, TENSOR_NEAR)
    check32("fmm32-tc-ragged-k2-r16", _rel(tc, ref))
