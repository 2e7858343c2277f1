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
fixed grid points g_k, which keep their areas, and the vorticity at g_k is
read off a local quadratic fitted to the moved particles near g_k:
  1. each moved particle belongs to the Voronoi cell of its nearest grid point
     (of two equally near ones, the one with the smaller index);
  2. the stencil of g_k is the set of grid points within `ring` edges of g_k in
     the grid's triangulation (ring 2: g_k, its neighbours and theirs), and the
     particles of their cells are the data;
  3. in gnomonic coordinates of the tangent plane at g_k scaled by h_k, the
     chord from g_k to its nearest neighbour in the triangulation,
     (u, v) = (x.e1, x.e2) / ((x.g_k) h_k) for an orthonormal pair e1, e2
     orthogonal to g_k, the quadratic c0 + c1 u + c2 v + c3 u^2 + c4 u v + c5 v^2
     is fitted by least squares with weights exp(-(u^2 + v^2)), and its value c0
     at g_k is the new zeta_k.
The fit reproduces quadratics in (u, v) exactly and is third-order accurate
for smooth fields; the tensor-product biquadratic of a structured grid has
no stencil on the icosahedral grid.  The choice of e1, e2 does not change c0.
"""
from __future__ import annotations

import numpy as np

from . import FMM, KERNEL_BIOT_SAVART, direct

# Planted mistakes for the pin tests (0 = none): 1 the Coriolis coupling with
# the wrong sign, 2 the second RK4 stage weighted 1 instead of 2, 3 the third
# stage started from the first stage's slope, 4 the last stage taken at
# t + dt/2, 5 the particle areas dropped from the weights; in the remeshing
# 6 orthographic instead of gnomonic coordinates, 7 a one-ring stencil, 8 the
# particle's starting grid point as its cell, 9 the u v term dropped, 10 the
# weights dropped.
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


def nearest_grid_point(grid, x):
    """Index of the grid point nearest to each x (Voronoi cell membership).
    Squared chords are formed as ((d0 d0 + d1 d1) + d2 d2) in FP64, and
    equally near grid points go to the smaller index: symmetric inputs (the
    icosahedral grid and RH wave share mirror symmetries) put particles
    exactly on cell boundaries.  The four nearest candidates of a k-d tree are
    compared in that arithmetic."""
    from scipy.spatial import cKDTree
    grid = np.asarray(grid, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    k = min(4, len(grid))
    cand = cKDTree(grid).query(x, k=k)[1].reshape(len(x), k)
    d = x[:, None, :] - grid[cand]
    d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    best = np.empty(len(x), dtype=np.int64)
    for i in range(len(x)):
        best[i] = min(zip(d2[i], cand[i]))[1]
    return best


def ring_stencil(offsets, nbrs, k: int, ring: int):
    """Grid points within `ring` triangulation edges of grid point k, ascending."""
    S = {int(k)}
    frontier = {int(k)}
    for _ in range(ring):
        new = set()
        for v in frontier:
            new.update(int(j) for j in nbrs[offsets[v]:offsets[v + 1]])
        frontier = new - S
        S |= new
    return sorted(S)


def tangent_basis(g):
    """An orthonormal pair e1, e2 orthogonal to the unit vector g."""
    a = np.array([0.0, 0.0, 1.0]) if abs(g[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    e1 = np.cross(a, g)
    e1 /= np.linalg.norm(e1)
    return e1, np.cross(g, e1)


def remesh_members(grid, offsets, nbrs, x, ring: int = 2):
    """For every grid point, the particles whose data enter its fit (steps 1-2
    of the remeshing), as lists of particle indices."""
    M = len(grid)
    cell = np.arange(len(x)) if _mutation == 8 else nearest_grid_point(grid, x)
    members = [[] for _ in range(M)]
    for p, c in enumerate(cell):
        members[c].append(p)
    r = 1 if _mutation == 7 else ring
    return [[p for s in ring_stencil(offsets, nbrs, k, r) for p in members[s]]
            for k in range(M)]


def neighbour_scale(grid, offsets, nbrs):
    """h_k: chord from each grid point to its nearest triangulation neighbour."""
    return np.array([min(np.linalg.norm(grid[j] - grid[k]) for j in nbrs[offsets[k]:offsets[k + 1]])
                     for k in range(len(grid))])


def remesh(grid, offsets, nbrs, x, f, ring: int = 2, points=None):
    """Vorticity at the grid points from the moved particles (x, f) by the
    local quadratic fit described in the module header.  Returns [M], or the
    values at the grid points listed in `points`."""
    grid = np.asarray(grid, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    Q = remesh_members(grid, offsets, nbrs, x, ring)
    h = neighbour_scale(grid, offsets, nbrs)
    ks = range(len(grid)) if points is None else points
    out = np.empty(len(ks))
    for i, k in enumerate(ks):
        g = grid[k]
        e1, e2 = tangent_basis(g)
        X = x[Q[k]]
        if _mutation == 6:
            u, v = (X @ e1) / h[k], (X @ e2) / h[k]
        else:
            den = (X @ g) * h[k]
            u, v = (X @ e1) / den, (X @ e2) / den
        cols = [np.ones_like(u), u, v, u * u, u * v, v * v]
        if _mutation == 9:
            cols[4] = np.zeros_like(u)
        sw = np.ones_like(u) if _mutation == 10 else np.exp(-0.5 * (u * u + v * v))
        c = np.linalg.lstsq(np.stack(cols, axis=1) * sw[:, None], f[Q[k]] * sw, rcond=None)[0]
        out[i] = c[0]
    return out


def remeshed_step(grid, offsets, nbrs, zeta, area, dt: float, omega: float, degree: int = 0,
                  theta: float = 0.7, N0=None, ring: int = 2):
    """One RK4 step from the grid points followed by remeshing onto them
    (Sec. 12): returns the new vorticity at the grid points."""
    x, z = rk4_step(grid, zeta, area, dt, omega, degree, theta, N0)
    return remesh(grid, offsets, nbrs, x, z, ring)
