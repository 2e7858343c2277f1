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

Remeshing (Sec. 12 remeshes at every step by local biquadratic interpolation,
without further detail).  Reading: after a step the particles return to the
fixed grid points g_k, which keep their areas, and the value at g_k of each
carried field is read off a local quadratic fitted to the moved particles
near g_k.  With h_k the chord from g_k to its nearest neighbour in the grid's
triangulation, an orthonormal pair e1, e2 orthogonal to g_k, and a particle
x with x.g_k > 0 in scaled gnomonic coordinates
    (u, v) = (x.e1, x.e2) / ((x.g_k) h_k),   s^2 = u^2 + v^2,
the data are the particles with s < S_C = 2.2, weighted by
(1 - s^2/S_C^2)^4, and c0 + c1 u + c2 v + c3 u^2 + c4 u v + c5 v^2 is fitted by
weighted least squares; the new value at g_k is c0.  The fit reproduces
quadratics in (u, v) exactly, is third-order accurate for smooth fields, and
-- the weights vanish smoothly at the edge of the data disc -- depends
continuously on the particle positions (a remeshing whose data set jumped
when a particle crossed a boundary would turn rounding-level asymmetries of
the velocity into truncation-level ones).  The tensor-product biquadratic of
a structured grid has no stencil on the icosahedral grid.  The choice of e1,
e2 does not change c0.
"""
from __future__ import annotations

import numpy as np

from . import FMM, KERNEL_BIOT_SAVART, direct

# Planted mistakes for the pin tests (0 = none): 1 the Coriolis coupling with
# the wrong sign, 2 the second RK4 stage weighted 1 instead of 2, 3 the third
# stage started from the first stage's slope, 4 the last stage taken at
# t + dt/2, 5 the particle areas dropped from the weights; in the remeshing
# 6 orthographic instead of gnomonic coordinates, 7 the h_k scaling dropped,
# 8 the u v term dropped, 9 the weights dropped.
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


S_C = 2.2  # radius of the data disc, in units of h_k


def tangent_basis(g):
    """An orthonormal pair e1, e2 orthogonal to the unit vector g."""
    a = np.array([0.0, 0.0, 1.0]) if abs(g[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    e1 = np.cross(a, g)
    e1 /= np.linalg.norm(e1)
    return e1, np.cross(g, e1)


def neighbour_scale(grid, offsets, nbrs):
    """h_k: chord from each grid point to its nearest triangulation neighbour."""
    return np.array([min(np.linalg.norm(grid[j] - grid[k]) for j in nbrs[offsets[k]:offsets[k + 1]])
                     for k in range(len(grid))])


def remesh_data(grid, h, x, k: int, tree=None):
    """Particles entering the fit at grid point k: (indices, u, v, weights)."""
    from scipy.spatial import cKDTree
    g = grid[k]
    hk = 1.0 if _mutation == 7 else h[k]
    tree = tree if tree is not None else cKDTree(x)
    # every particle with s < S_C lies within this chord of g_k
    r = 2.0 * np.sin(0.5 * np.arctan(S_C * hk)) * (1.0 + 1e-9)
    Q = np.asarray(tree.query_ball_point(g, r), dtype=np.int64)
    X = x[Q]
    e1, e2 = tangent_basis(g)
    dot = X @ g
    if _mutation == 6:
        u, v = (X @ e1) / hk, (X @ e2) / hk
    else:
        den = np.where(dot > 0, dot * hk, 1.0)
        u, v = (X @ e1) / den, (X @ e2) / den
    s2 = u * u + v * v
    keep = (dot > 0) & (s2 < S_C * S_C)
    w = np.ones(int(keep.sum())) if _mutation == 9 else (1.0 - s2[keep] / (S_C * S_C)) ** 4
    return Q[keep], u[keep], v[keep], w


def remesh(grid, offsets, nbrs, x, f, points=None):
    """Values at the grid points from the moved particles x carrying f ([M]
    or [nfield, M]) by the local quadratic fit described in the module
    header.  Returns f's shape with M replaced by the grid points (or by the
    grid points listed in `points`)."""
    from scipy.spatial import cKDTree
    grid = np.asarray(grid, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    F = f.reshape(-1, f.shape[-1])
    h = neighbour_scale(grid, offsets, nbrs)
    tree = cKDTree(x)
    ks = range(len(grid)) if points is None else points
    out = np.empty((len(F), len(ks)))
    for i, k in enumerate(ks):
        Q, u, v, w = remesh_data(grid, h, x, k, tree)
        cols = [np.ones_like(u), u, v, u * u, u * v, v * v]
        if _mutation == 8:
            cols[4] = np.zeros_like(u)
        sw = np.sqrt(w)
        c = np.linalg.lstsq(np.stack(cols, axis=1) * sw[:, None], (F[:, Q] * sw).T,
                            rcond=None)[0]
        out[:, i] = c[0]
    return out[0] if f.ndim == 1 else out


def remeshed_step(grid, offsets, nbrs, zeta, area, dt: float, omega: float, degree: int = 0,
                  theta: float = 0.7, N0=None, tracer=None):
    """One RK4 step from the grid points followed by remeshing onto them
    (Sec. 12): returns the new vorticity at the grid points, or (vorticity,
    tracer) with a passive tracer, which the particles carry unchanged
    (dq/dt = 0 along paths) and which is remeshed with the vorticity."""
    x, z = rk4_step(grid, zeta, area, dt, omega, degree, theta, N0)
    if tracer is None:
        return remesh(grid, offsets, nbrs, x, z)
    out = remesh(grid, offsets, nbrs, x, np.stack([z, np.asarray(tracer, dtype=np.float64)]))
    return out[0], out[1]


def tracer_properties(q, area):
    """Tracer mass m = sum q_i A_i and bound q_max = max |q_i| (Sec. 12)."""
    q = np.asarray(q)
    return float(np.sum(q * np.asarray(area))), float(np.max(np.abs(q)))
