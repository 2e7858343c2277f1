"""Pins of the oracle's vortex method for the barotropic vorticity equation
(Sec. 2.3, Eq. BVE_ODEs; Sec. 12: RK4, Omega = 2 pi per day, dt = 0.01 day).

What fixes the answer without the oracle: the classical RK4 error falls 16x
per halving of dt; the ODEs carry zeta + 2 Omega z with each particle
(Eq. BVE); a solid-body vorticity 2 w z rotates every particle about the z
axis at angular speed w; the RH wave of Eq. RH_initial is stationary, so
zeta_i(t) = zeta_0(x_i(t)) and E_zeta (Eq. bveerr) falls like the midpoint
rule's O(dphi^2), about 4x per icosahedral level; the Gaussian vortex of
Eq. Gaussian_ic has zero total vorticity (its background is pi/16 to the
printed digits) and its core drifts north-west (Sec. 12).  Each planted
mistake in the RK4 integrator fails at least one of these.
"""
import math

import numpy as np
import pytest

import oracle.bve as B
from paper_2508_13550_gb300 import inputs as I

OMEGA = I.BVE_OMEGA


def _order_ratios():
    x, z, A = I.workload_bve(2)
    T = 0.4
    ref = B.integrate(x, z, A, T / 128, 128, OMEGA)
    errs = []
    for n in (8, 16, 32):
        xs, zs = B.integrate(x, z, A, T / n, n, OMEGA)
        errs.append(max(np.abs(xs - ref[0]).max(), np.abs(zs - ref[1]).max()))
    return [errs[i] / errs[i + 1] for i in range(2)]


def _pin_fourth_order():
    return all(14.0 < r < 18.0 for r in _order_ratios())


def _pin_absolute_vorticity():
    x, z, A = I.workload_bve(3)
    xs, zs = B.integrate(x, z, A, I.BVE_DT, 5, OMEGA)
    drift = np.abs((zs + 2 * OMEGA * xs[:, 2]) - (z + 2 * OMEGA * x[:, 2])).max()
    return drift < 1e-7 * np.abs(zs - z).max()


def _rh_errors(levels=(2, 3, 4), steps=10):
    out = []
    for lev in levels:
        x, z, A = I.workload_bve(lev)
        xs, zs = B.integrate(x, z, A, I.BVE_DT, steps, OMEGA)
        out.append(B.vorticity_error(zs, I.rossby_haurwitz_vorticity(xs), A))
    return out


def _pin_rh_stationary():
    e = _rh_errors()
    return e[-1] < 5e-3 and all(3.0 < e[i] / e[i + 1] < 5.0 for i in range(len(e) - 1))


def test_rk4_is_fourth_order():
    r = _order_ratios()
    print("\nerror ratios per halving of dt:", r)
    assert all(14.0 < x < 18.0 for x in r)


def test_absolute_vorticity_is_carried():
    assert _pin_absolute_vorticity()


def test_solid_body_rotation():
    """zeta = 2 w z with Omega = 0: psi = w z, u = w e_z x x, each particle
    turns by w t about the z axis at fixed z (up to the midpoint rule's
    quadrature error on the level-4 grid)."""
    x, _, A = I.workload_bve(4)
    w = 0.7
    z0 = 2 * w * x[:, 2]
    xs, zs = B.integrate(x, z0, A, 0.05, 4, 0.0)
    ang = np.arctan2(xs[:, 1], xs[:, 0]) - np.arctan2(x[:, 1], x[:, 0])
    ang = (ang + np.pi) % (2 * np.pi) - np.pi
    m = np.abs(x[:, 2]) < 0.9
    assert abs(np.median(ang[m]) - w * 0.2) < 2e-3 * w * 0.2
    assert np.abs(ang[m] - w * 0.2).max() < 0.02 * w * 0.2
    assert np.abs(xs[:, 2] - x[:, 2]).max() < 1e-3
    assert np.array_equal(zs, z0)


def test_rh_wave_stationary_error_converges_second_order():
    e = _rh_errors()
    print("\nE_zeta(0.1 day), icosahedral levels 2, 3, 4:", e)
    assert e[-1] < 5e-3
    for i in range(len(e) - 1):
        assert 3.0 < e[i] / e[i + 1] < 5.0


def test_fmm_velocity_error_below_discretisation():
    """Sec. 12: with MAC 0.7 and n = 6 the CSFMM error is negligible next to
    the discretisation error: one step with the CSFMM velocity matches the
    direct-sum step far below E_zeta."""
    x, z, A = I.workload_bve(4)
    xd, zd = B.rk4_step(x, z, A, I.BVE_DT, OMEGA)
    xf, zf = B.rk4_step(x, z, A, I.BVE_DT, OMEGA, degree=6, theta=0.7)
    assert np.abs(xf - xd).max() < 1e-6
    assert B.vorticity_error(zf, zd, A) < 1e-6
    assert np.allclose(np.linalg.norm(xf, axis=1), 1.0, atol=1e-15)


def test_gaussian_vortex_zero_total_vorticity():
    """int 4 pi exp(-16 |x - x_c|^2) dS = (pi^2/4)(1 - e^-64), so the
    background that zeroes the total is pi/16 = 0.19634954...; the printed
    0.196353 agrees to 4e-6, and the midpoint sum on the level-5 grid is
    within its quadrature error of zero."""
    assert abs(math.pi / 16 - 0.196353) < 5e-6
    x, z, A = I.workload_bve(5, "gaussian")
    assert abs(np.sum(z * A)) < 1e-3 * np.sum(np.abs(z) * A)


def test_gaussian_vortex_drifts_north_west():
    """Sec. 12: the core of the Gaussian vortex moves to the north-west."""
    x, z, A = I.workload_bve(4, "gaussian")
    xs, zs = B.integrate(x, z, A, I.BVE_DT, 30, OMEGA)

    def core(p, f):
        w = np.maximum(f - 0.5 * f.max(), 0.0) * A
        c = (w[:, None] * p).sum(0)
        c /= np.linalg.norm(c)
        return math.asin(c[2]), math.atan2(c[1], c[0])

    lat0, lon0 = core(x, z)
    lat1, lon1 = core(xs, zs)
    assert lat1 > lat0 + math.radians(3)
    assert lon1 < lon0 - math.radians(1)


MUTATIONS = {1: "Coriolis coupling sign", 2: "RK4 weight of stage 2", 3: "stage 3 slope",
             4: "last stage time", 5: "areas dropped"}


@pytest.mark.parametrize("m", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(m):
    B.set_mutation(m)
    try:
        caught = not (_pin_fourth_order() and _pin_absolute_vorticity() and _pin_rh_stationary())
    finally:
        B.set_mutation(0)
    assert caught, MUTATIONS[m]
