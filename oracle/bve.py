"""Vortex method for the barotropic vorticity equation, CPU oracle side.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.

Sec. 2.3, Eq. BVE_ODEs: particles x_i on the unit sphere with relative
vorticity zeta_i and fixed areas A_i obey
    dx_i/dt = sum_{j != i} K_BS(x_i, x_j) zeta_j A_j,
    dzeta_i/dt = -2 Omega dz_i/dt,
so that the absolute vorticity zeta + 2 Omega z of each particle is constant
(Eq. BVE, Coriolis parameter f = 2 Omega z).  Sec. 12 integrates them with the
classical fourth-order Runge-Kutta method.  The velocity comes from the
oracle's direct sum (degree 0) or its CSFMM (a tree built at every stage's
positions).  The paper is silent on how a Runge-Kutta stage that leaves the
sphere is handled; here the stage positions and the step result are
projected radially back onto the unit sphere, where K_BS is defined (the
exact flow is tangent to the sphere, so this keeps the method's order).
Remeshing is not part of the step.
"""
from __future__ import annotations

import numpy as np

from . import FMM, KERNEL_BIOT_SAVART, direct

# Planted mistakes for the pin tests (0 = none): 1 the Coriolis coupling with
# the wrong sign, 2 the second RK4 stage weighted 1 instead of 2, 3 the third
# stage started from the first stage's slope, 4 the last stage taken at
# t + dt/2, 5 the particle areas dropped from the weights.
_mutation = 0


def set_mutation(m: int) -> None:
    global _mutation
    _mutation = int(m)


def velocity(x, zeta, area, degree: int = 0, theta: float = 0.7, N0: int | None = None):
    """dx/dt of Eq. BVE_ODEs at positions x: the Biot-Savart sum with weights
    zeta_j A_j, by direct summation (degree 0) or the CSFMM.  Returns [N, 3]."""
    w = np.asarray(zeta) * (1.0 if _mutation == 5 else np.asarray(area))
    if degree == 0:
        return direct(x, KERNEL_BIOT_SAVART, w)[0]
    leaf = N0 if N0 is not None else max(1, 4 * degree * degree)
    return FMM(x, degree, theta, leaf).evaluate(KERNEL_BIOT_SAVART, w)[0]


def project(y):
    """Radial projection onto the unit sphere."""
    return y / np.linalg.norm(y, axis=1, keepdims=True)


def rhs(x, zeta, area, omega: float, degree: int = 0, theta: float = 0.7, N0=None):
    """Right-hand side of Eq. BVE_ODEs: (dx/dt [N,3], dzeta/dt [N])."""
    u = velocity(x, zeta, area, degree, theta, N0)
    return u, (2.0 if _mutation == 1 else -2.0) * omega * u[:, 2]


def rk4_step(x, zeta, area, dt: float, omega: float, degree: int = 0, theta: float = 0.7,
             N0=None):
    """One classical RK4 step of Eq. BVE_ODEs (stages at t, t + dt/2, t + dt/2,
    t + dt; weights 1/6, 2/6, 2/6, 1/6), positions projected onto the sphere
    at every stage.  Returns (x, zeta) at t + dt."""
    x = np.asarray(x, dtype=np.float64)
    zeta = np.asarray(zeta, dtype=np.float64)
    k1x, k1z = rhs(x, zeta, area, omega, degree, theta, N0)
    k2x, k2z = rhs(project(x + 0.5 * dt * k1x), zeta + 0.5 * dt * k1z, area, omega, degree,
                   theta, N0)
    s2x, s2z = (k1x, k1z) if _mutation == 3 else (k2x, k2z)
    k3x, k3z = rhs(project(x + 0.5 * dt * s2x), zeta + 0.5 * dt * s2z, area, omega, degree,
                   theta, N0)
    h4 = 0.5 * dt if _mutation == 4 else dt
    k4x, k4z = rhs(project(x + h4 * k3x), zeta + h4 * k3z, area, omega, degree, theta, N0)
    b2 = 1.0 if _mutation == 2 else 2.0
    x_new = project(x + (dt / 6.0) * (k1x + b2 * k2x + 2 * k3x + k4x))
    zeta_new = zeta + (dt / 6.0) * (k1z + b2 * k2z + 2 * k3z + k4z)
    return x_new, zeta_new


def integrate(x, zeta, area, dt: float, steps: int, omega: float, degree: int = 0,
              theta: float = 0.7, N0=None):
    """steps RK4 steps from (x, zeta)."""
    for _ in range(steps):
        x, zeta = rk4_step(x, zeta, area, dt, omega, degree, theta, N0)
    return x, zeta


def vorticity_error(zeta, zeta_exact, area):
    """E_zeta of Eq. bveerr: the area-weighted relative l2 error
    sqrt(sum (zeta_i - zeta_0(x_i))^2 A_i / sum zeta_0(x_i)^2 A_i)."""
    d = np.asarray(zeta) - np.asarray(zeta_exact)
    A = np.asarray(area)
    return float(np.sqrt(np.sum(d * d * A) / np.sum(np.asarray(zeta_exact) ** 2 * A)))
