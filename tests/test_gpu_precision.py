"""Accuracy of the FP32-bulk form on uniform grids, against the oracle's FP64
direct sum on sampled targets.

On an equiangular cubed-sphere grid every leaf holds the same local point
pattern, so any constant rounded to FP32 once and reused in every cell (the
Lagrange rows of the points, the M2M matrices, a cell's weight total) turns
into a bias of the whole potential instead of averaging out.  These bars
were measured on GB300 after those errors were removed (Newtonian, m = 256,
n = 8: E = 1.5e-8, bias -1.2e-8; Poisson Y43: E = 1.7e-7, bias 7e-9); with
FP32 M2M arithmetic the Newtonian bias was +2.8e-8, with round-to-nearest
rows and FP32 M2M +1.6e-8 and +6e-8 at N = 6.3M, and with FP32 per-tile
weight totals the Poisson bias was +6e-8.
"""
import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I
from gpu_util import cuda_or_skip, dev
from fp32_bars import check as check32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def C():
    from paper_2508_13550_gb300 import csfmm
    return csfmm


def errors(torch, C, pts, kernel, w, n, N0, nsample=768):
    """(E, bias) of the FP32-bulk FMM against the oracle direct sum on
    seeded sampled targets: E = |f - ds|_2 / |ds|_2, bias = sum(f - ds) /
    sum|ds|."""
    tg = np.sort(np.random.default_rng(5).choice(len(pts), nsample, replace=False))
    ds = O.direct(pts, kernel, w, tg)[0, :, 0]
    P = C.plan_create(dev(torch, pts), kernel, n, 0.7, N0, precision=C.FP32_BULK)
    out = C.evaluate(P, dev(torch, np.atleast_2d(w)))
    torch.cuda.synchronize()
    C.plan_sync(P)
    f = out[0, :, 0].cpu().numpy()[tg]
    C.plan_destroy(P)
    d = f - ds
    return float(np.linalg.norm(d) / np.linalg.norm(ds)), float(d.sum() / np.abs(ds).sum())


def test_fp32_bulk_newton_uniform_grid_unbiased(torch, C):
    pts, A = I.cubed_sphere_grid(256)
    w = I.land_mask_field(pts, I.MASTER_SEED + 3) * A
    e, bias = errors(torch, C, pts, O.KERNEL_NEWTON, w, 8, 256)
    print(f"\nNewtonian m=256 n=8: E={e:.3e} bias={bias:.3e}")
    check32("fmm32-newton-land-m256-n8", e)
    assert abs(bias) < 2.2e-8


def test_fp32_bulk_poisson_uniform_grid(torch, C):
    pts, A, w, _ = I.workload_poisson_y43(256)
    e, bias = errors(torch, C, pts, O.KERNEL_LAPLACE, w, 8, 256)
    print(f"\nPoisson Y43 m=256 n=8: E={e:.3e} bias={bias:.3e}")
    check32("fmm32-poisson-y43-m256-n8", e)
    assert abs(bias) < 3e-8


def test_fp32_bulk_biharmonic_against_direct(torch, C):
    """Biharmonic kernel (Eq. G_B) in the FP32-bulk form: the FP32 dilogarithm
    (two MUFU logarithms and a Bernoulli series) keeps the error against the
    FP64 direct sum near FP32 rounding."""
    pts, A = I.cubed_sphere_grid(128)
    w = I.land_mask_field(pts, 21) * A
    e, bias = errors(torch, C, pts, O.KERNEL_BIHARMONIC, w, 8, 256)
    print(f"\nbiharmonic m=128 n=8: E={e:.3e} bias={bias:.3e}")
    check32("fmm32-biharmonic-land-m128-n8", e)
