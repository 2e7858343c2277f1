"""GPU parity for separate target and source sets (csfmm_plan_create_targets;
Sec. 1) through the C ABI against the oracle on the same seeded inputs.

Bars: FP64 CSFMM and CSTC against the oracle's CSFMM and CSTC on the same
tree, relative l2 <= 1e-12; FP32 bulk against the oracle direct sum at most
the per-case bar of fp32_bars.py (about 4x the error measured on GB300; the
Biot-Savart velocity, whose sum cancels, has the largest);
K = 1 reproduces sum_j w_j at every target.
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


SETS = [
    ("random 3000 -> random 1000", lambda: (I.random_sphere_points(3000, 41),
                                            I.random_sphere_points(1000, 42)), 6, 0.7, 40),
    ("icosahedral L4 -> lat-lon L4", lambda: (I.icosahedral_grid(4)[0], I.latlon_grid(4)[0]),
     5, 0.7, 30),
    ("random 500 -> 1 target", lambda: (I.random_sphere_points(500, 43),
                                        I.random_sphere_points(1, 44)), 4, 0.8, 10),
    ("1 source -> random 300", lambda: (I.random_sphere_points(1, 45),
                                        I.random_sphere_points(300, 46)), 3, 0.7, 8),
]


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("name,mk,n,theta,N0", SETS)
def test_fp64_matches_oracle(torch, C, name, mk, n, theta, N0, kernel):
    src, tgt = mk()
    W = np.random.default_rng(47).standard_normal((2, len(src))) / len(src)
    ref = O.fmm_targets(src, tgt, n, theta, N0, kernel, W)
    P = C.plan_create_targets(dev(torch, src), dev(torch, tgt), kernel, n, theta, N0)
    got = C.evaluate(P, dev(torch, W)).cpu().numpy()
    assert got.shape == ref.shape
    assert rel(got, ref) < 1e-12, (name, kernel, rel(got, ref))


@pytest.mark.parametrize("name,mk,n,theta,N0", SETS[:2])
def test_cstc_matches_oracle(torch, C, name, mk, n, theta, N0):
    src, tgt = mk()
    w = np.random.default_rng(48).standard_normal(len(src))
    ref = O.fmm_targets(src, tgt, n, theta, N0, O.KERNEL_LAPLACE, w, cstc=True)
    P = C.plan_create_targets(dev(torch, src), dev(torch, tgt), 0, n, theta, N0)
    got = C.evaluate_cstc(P, dev(torch, np.atleast_2d(w))).cpu().numpy()
    assert rel(got, ref) < 1e-12


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_fp32_bulk_against_direct(torch, C, kernel):
    src, tgt = I.random_sphere_points(20000, 49), I.random_sphere_points(3000, 50)
    # a land-mask density (positive, as the paper's fields): random signs would
    # measure FP32 rounding against a sum that cancels
    w = I.land_mask_field(src, 51) / len(src)
    ds = O.direct_targets(src, kernel, w, tgt)
    P = C.plan_create_targets(dev(torch, src), dev(torch, tgt), kernel, 10, 0.5, 200,
                              precision=C.FP32_BULK)
    got = C.evaluate(P, dev(torch, np.atleast_2d(w))).cpu().numpy()
    print(f"\nkernel {kernel} FP32 bulk at separate targets: {rel(got, ds):.2e}")
    check32(f"fmm32-targets-k{kernel}", rel(got, ds))


def test_constant_kernel_and_host_entry(torch, C):
    src, tgt = I.random_sphere_points(4000, 52), I.random_sphere_points(900, 53)
    w = np.random.default_rng(54).standard_normal((3, len(src)))
    # FP32 bulk rounds every weight once (relative 6e-8): bound 1e-7 sum|w|
    for prec, tol in ((C.FP64, 1e-13), (C.FP32_BULK, 1e-7)):
        P = C.plan_create_targets(dev(torch, src), dev(torch, tgt), C.KERNEL_ONE, 3, 0.7, 16,
                                  precision=prec, max_nrhs=2)
        got = C.evaluate(P, dev(torch, w)).cpu().numpy()[:, :, 0]
        assert np.abs(got - w.sum(1)[:, None]).max() < tol * np.abs(w).sum()
        host = C.evaluate_host(P, w)
        assert np.array_equal(host, C.evaluate(P, dev(torch, w)).cpu().numpy())
