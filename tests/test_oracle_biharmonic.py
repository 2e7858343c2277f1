"""Pins of the oracle's biharmonic kernel G_B(x, y) = (1/4pi) dilog((1 + x.y)/2)
(Sec. 2, Eq. G_B), a NEXT-row kernel: the dilogarithm against independent
evaluations, and the Funk-Hecke eigenvalues 1/(n^2 (n+1)^2) of the spherical
biharmonic operator (Delta^2 Y_n = n^2 (n+1)^2 Y_n, Sec. 2)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I


def test_dilog_special_values_and_scipy():
    assert abs(O.dilog(1.0) - math.pi ** 2 / 6) < 1e-15
    assert abs(O.dilog(0.5) - (math.pi ** 2 / 12 - math.log(2) ** 2 / 2)) < 1e-15
    assert O.dilog(0.0) == 0.0
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    for x in np.linspace(1e-3, 1.0, 997):
        ref = float(mpmath.polylog(2, mpmath.mpf(float(x))))
        assert abs(O.dilog(x) - ref) <= 2e-15 * abs(ref), x
    # scipy's spence(z) = Li2(1 - z) loses digits for z near 1; away from it
    sp = pytest.importorskip("scipy.special")
    for x in np.linspace(0.05, 1.0, 96):
        assert abs(O.dilog(x) - sp.spence(1.0 - x)) <= 1e-14 * O.dilog(x), x


def test_dilog_power_series_near_zero():
    for x in (1e-12, 1e-8, 1e-4, 1e-2):
        ref = sum(x ** k / k ** 2 for k in range(1, 30))
        assert abs(O.dilog(x) - ref) <= 1e-15 * ref


@pytest.mark.parametrize("n,m", [(1, 0), (2, 1), (4, 3)])
def test_biharmonic_funk_hecke_eigenvalue_second_order(n, m):
    """sum_j G_B(x_i, x_j) Y(x_j) A_j -> Y(x_i) / (n^2 (n+1)^2): second order in
    the spacing (the omitted i = j term, G_B(x, x) = pi/24, is O(A_i))."""
    lam = 1.0 / (n * n * (n + 1) ** 2)
    errs = []
    for mm in (16, 32, 64):
        pts, A = I.cubed_sphere_grid(mm)
        y = I.real_sph_harm(n, m, pts)
        ds = O.direct(pts, O.KERNEL_BIHARMONIC, y * A)[0, :, 0]
        errs.append(O.rel_l2(ds, lam * y, A))
    assert errs[0] > 3.5 * errs[1] > 12.0 * errs[2], errs


def test_biharmonic_direct_sum_rotation_invariant():
    pts, A = I.cubed_sphere_grid(16)
    w = I.land_mask_field(pts, 4) * A
    R = I.random_rotation(9)
    a = O.direct(pts, O.KERNEL_BIHARMONIC, w)
    b = O.direct(pts @ R.T, O.KERNEL_BIHARMONIC, w)
    assert O.rel_l2(a, b) < 1e-13


def test_biharmonic_fmm_and_cstc_converge_to_direct_sum():
    pts, A = I.cubed_sphere_grid(8)
    w = I.real_sph_harm(4, 3, pts) * A
    ds = O.direct(pts, O.KERNEL_BIHARMONIC, w)[0, :, 0]
    f = O.FMM(pts, 14, 0.5, 16)
    assert O.rel_l2(f.evaluate(O.KERNEL_BIHARMONIC, w)[0, :, 0], ds, A) < 1e-11
    assert O.rel_l2(f.evaluate_cstc(O.KERNEL_BIHARMONIC, w)[0, :, 0], ds, A) < 1e-11
    pts, A = I.cubed_sphere_grid(32)
    w = I.land_mask_field(pts, 5) * A
    ds = O.direct(pts, O.KERNEL_BIHARMONIC, w)[0, :, 0]
    e = [O.rel_l2(O.FMM(pts, n, 0.7, 64).evaluate(O.KERNEL_BIHARMONIC, w)[0, :, 0], ds)
         for n in (2, 4, 6, 8)]
    assert all(a > 5 * b for a, b in zip(e, e[1:])), e
