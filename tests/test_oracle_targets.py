"""Pins of the oracle for separate target and source sets (Sec. 1: the scheme
accommodates targets that are not the sources).

What fixes the answer: with K = 1 every interaction is exact, so the CSFMM
returns sum_j w_j at every target, which fails if a source is missed or
counted twice or a target's zero weight leaks in; at targets off the source
grid the direct sum of Y_n^m A approximates the Funk-Hecke potential
Y_n^m / (n (n + 1)) to the midpoint rule's accuracy; and the CSFMM and CSTC
at separate targets converge to the direct sum with the degree.
"""
import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I


def test_constant_kernel_sums_every_source_once():
    src = I.random_sphere_points(2500, 31)
    tgt = I.random_sphere_points(700, 32)
    w = np.random.default_rng(33).standard_normal(len(src))
    for cstc in (False, True):
        out = O.fmm_targets(src, tgt, 3, 0.7, 12, O.KERNEL_ONE, w, cstc=cstc)[0, :, 0]
        assert np.abs(out - w.sum()).max() < 1e-11


def test_funk_hecke_at_off_grid_targets():
    pts, A = I.cubed_sphere_grid(48)
    Y = I.real_sph_harm(4, 3, pts)
    tgt = I.random_sphere_points(400, 34)
    got = O.direct_targets(pts, O.KERNEL_LAPLACE, Y * A, tgt)[0, :, 0]
    exact = I.real_sph_harm(4, 3, tgt) / 20.0
    err = np.linalg.norm(got - exact) / np.linalg.norm(exact)
    print(f"\nFunk-Hecke at 400 random targets, m = 48: rel err {err:.2e}")
    assert err < 2e-3


@pytest.mark.parametrize("kernel", [O.KERNEL_LAPLACE, O.KERNEL_BIOT_SAVART, O.KERNEL_NEWTON])
def test_fmm_at_targets_converges_to_direct(kernel):
    src = I.random_sphere_points(3000, 35)
    tgt = I.random_sphere_points(642, 36)
    w = np.random.default_rng(37).standard_normal(len(src)) / len(src)
    ds = O.direct_targets(src, kernel, w, tgt)
    errs = []
    for n in (4, 8, 12):
        fs = O.fmm_targets(src, tgt, n, 0.7, 40, kernel, w)
        errs.append(np.linalg.norm(fs - ds) / np.linalg.norm(ds))
    print(f"\nkernel {kernel}: errors n = 4, 8, 12: {errs}")
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-7
