"""Pins of the oracle's SAL kernel: the bracket of Eq. G_SAL_approx,
(1 - b0)/gamma - (a1 - b1) ln(gamma/2 + gamma^2/4) with the paper's Love
number fit a1 = -2.7, b0 = -6.21196, b1 = 6.1 (Sec. 2.4), gamma = |x - y|.

What fixes it: by the Legendre sums the paper uses (Eq. Legendre),
1/gamma = sum_n P_n and -ln(gamma/2 + gamma^2/4) = sum_{n>=1} P_n / n, so by
Funk-Hecke the kernel has the eigenvalue
    lambda_n = 4 pi ((1 - b0) + (a1 - b1)/n) / (2n + 1)
on degree-n harmonics -- the paper's approximation (1 + k'_n - h'_n) of the
SAL multipliers.  Its log part alone (the kernel minus (1 - b0) times the
Newtonian kernel) has eigenvalue 4 pi (a1 - b1)/(n (2n + 1)), and the direct
sum converges to both with the grid; a flipped sign or a dropped factor of
the log term fails them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I

A1, B0, B1 = -2.7, -6.21196, 6.1


def lam(n):
    return 4 * math.pi * ((1 - B0) + (A1 - B1) / n) / (2 * n + 1)


def _errors(n, m_list, log_part):
    out = []
    for m in m_list:
        pts, A = I.cubed_sphere_grid(m)
        Y = I.real_sph_harm(n, 2 if n >= 2 else 0, pts)
        w = Y * A
        phi = O.direct(pts, O.KERNEL_SAL, w)[0, :, 0]
        if log_part:
            phi = phi - (1 - B0) * O.direct(pts, O.KERNEL_NEWTON, w)[0, :, 0]
            ex = 4 * math.pi * (A1 - B1) / (n * (2 * n + 1)) * Y
        else:
            ex = lam(n) * Y
        out.append(O.rel_l2(phi, ex, A))
    return out


@pytest.mark.parametrize("n", [1, 4])
def test_log_part_eigenvalue_converges(n):
    e = _errors(n, (32, 64), log_part=True)
    print(f"\nSAL log part, n = {n}: E = {e}")
    assert e[1] < 1e-2 and e[0] / e[1] > 3.0  # measured 3.5x per halving of h


def test_full_kernel_eigenvalue():
    """The 1/gamma part makes the punctured midpoint rule first order (the
    omitted self cell carries O(h) of the Newtonian integral)."""
    e = _errors(4, (32, 64), log_part=False)
    print(f"\nSAL kernel, n = 4: E = {e} (lambda_4 = {lam(4):.4f})")
    assert e[1] < 0.1 and e[0] / e[1] > 1.8


def test_fmm_high_degree_equals_direct():
    pts, A = I.cubed_sphere_grid(12)
    w = np.random.default_rng(3).standard_normal(len(pts)) * A
    ds = O.direct(pts, O.KERNEL_SAL, w)[0, :, 0]
    fs = O.FMM(pts, 14, 0.7, 16).evaluate(O.KERNEL_SAL, w)[0, :, 0]
    assert np.linalg.norm(fs - ds) / np.linalg.norm(ds) < 1e-11
