"""GPU parity of the SAL kernel (CSFMM_KERNEL_SAL: the bracket of Eq.
G_SAL_approx with the paper's Love number fit) through the C ABI against the
oracle on the same seeded inputs.

Bars: FP64 CSFMM and CSTC vs the oracle's, relative l2 <= 1e-12; FP64 direct
sum vs the oracle's <= 1e-13; FP32 bulk vs the oracle's FP64 direct sum (or
its FMM on the same tree) at most the per-case bar of fp32_bars.py (about 4x
the error measured on GB300); several right-hand sides against one at a time.
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


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


CASES = [
    ("cubed m=24, Y43, n=8 N0=64", lambda: I.cubed_sphere_grid(24)[0], 8, 0.7, 64),
    ("random 3000, n=6 N0=30", lambda: I.random_sphere_points(3000, 61), 6, 0.7, 30),
    ("icosahedral L4, n=5 N0=20 MAC 0.5", lambda: I.icosahedral_grid(4)[0], 5, 0.5, 20),
]


@pytest.mark.parametrize("name,mk,n,theta,N0", CASES)
def test_fp64_fmm_cstc_direct_match_oracle(torch, C, name, mk, n, theta, N0):
    pts = mk()
    W = np.random.default_rng(62).standard_normal((2, len(pts))) / len(pts)
    f = O.FMM(pts, n, theta, N0)
    P = C.plan_create(dev(torch, pts), C.KERNEL_SAL, n, theta, N0)
    got = C.evaluate(P, dev(torch, W)).cpu().numpy()
    assert rel(got, f.evaluate(O.KERNEL_SAL, W)) < 1e-12
    gc = C.evaluate_cstc(P, dev(torch, W)).cpu().numpy()
    assert rel(gc, f.evaluate_cstc(O.KERNEL_SAL, W)) < 1e-12
    ds = C.direct(dev(torch, pts), C.KERNEL_SAL, dev(torch, W)).cpu().numpy()
    assert rel(ds, O.direct(pts, O.KERNEL_SAL, W)) < 1e-13


def test_fp32_bulk_against_fp64_direct(torch, C):
    pts, A = I.cubed_sphere_grid(128)
    w = I.land_mask_field(pts, 63) * A
    tg = np.sort(np.random.default_rng(64).choice(len(pts), 768, replace=False))
    ds = O.direct(pts, O.KERNEL_SAL, w, tg)[0, :, 0]
    P = C.plan_create(dev(torch, pts), C.KERNEL_SAL, 8, 0.7, 256, precision=C.FP32_BULK)
    got = C.evaluate(P, dev(torch, np.atleast_2d(w))).cpu().numpy()[0, tg, 0]
    d32 = C.direct(dev(torch, pts), C.KERNEL_SAL, dev(torch, np.atleast_2d(w)),
                   precision=C.FP32_BULK).cpu().numpy()[0, tg, 0]
    print(f"\nSAL FP32 bulk m=128 n=8: FMM {rel(got, ds):.2e}, direct {rel(d32, ds):.2e}")
    check32("fmm32-sal-land-m128-n8", rel(got, ds))
    check32("direct32-sal-land-m128", rel(d32, ds))


def test_fp32_multi_rhs_matches_single(torch, C):
    pts = I.random_sphere_points(20000, 65)
    W = np.random.default_rng(66).random((8, len(pts))) / len(pts)
    P = C.plan_create(dev(torch, pts), C.KERNEL_SAL, 7, 0.7, 80, precision=C.FP32_BULK,
                      max_nrhs=8)
    allr = C.evaluate(P, dev(torch, W)).cpu().numpy()
    ref = O.FMM(pts, 7, 0.7, 80).evaluate(O.KERNEL_SAL, W[[0, 5]])
    for k, r in enumerate((0, 5)):
        one = C.evaluate(P, dev(torch, W[r:r + 1])).cpu().numpy()[0]
        check32("fmm32-sal-chunk-vs-single", rel(allr[r], one))
        check32("fmm32-sal-multi-vs-oracle-fmm", rel(allr[r], ref[k]))
