"""Pins of the oracle's remeshing (Sec. 12: remeshing at every step by local
interpolation; the reading -- nearest-grid-point cells, a two-ring stencil of
the triangulation, a Gaussian-weighted quadratic least-squares fit in scaled
gnomonic coordinates -- is stated in oracle/bve.py).

What fixes the answer without the oracle: a quadratic in the gnomonic
coordinates of g_k is reproduced exactly at g_k whatever the particles'
positions; the stencil of a hexagonal vertex has 1 + 6 + 12 grid points and
of a pentagonal one 1 + 5 + 10, and its data are the particles whose nearest
grid point (brute force) lies in it; the remeshing error of a smooth field
falls third-order with the grid spacing; the icosahedral triangulation is the
Delaunay triangulation (convex hull) of its vertices, so a greedy walk ends at
the nearest grid point; and with remeshing the RH wave's E_zeta keeps falling
with N as Sec. 12 reports.  Planted mistakes 6-10 each fail one of these.
"""
import numpy as np
import pytest

import oracle.bve as B
from paper_2508_13550_gb300 import inputs as I

OMEGA = I.BVE_OMEGA


def moved(level, steps=1):
    """Grid, adjacency and the particles after RK4 steps of the RH wave."""
    x, z, A, off, nb = I.workload_bve(level, with_adjacency=True)
    xs, zs = B.integrate(x, z, A, I.BVE_DT, steps, OMEGA)
    return x, off, nb, xs, zs, A, z


def _pin_quadratic_exact():
    x, off, nb, xs, _, _, _ = moved(3, steps=10)
    rng = np.random.default_rng(4)
    h = B.neighbour_scale(x, off, nb)
    for k in (0, 7, 100, 331, 641):  # 0 and 7: pentagonal vertices
        g = x[k]
        a = np.array([0.3, 0.8, -0.5]) if abs(g[0]) < 0.9 else np.array([0.0, 1.0, 0.2])
        e1 = a - (a @ g) * g
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(g, e1)
        den = (xs @ g) * h[k]
        u, v = (xs @ e1) / den, (xs @ e2) / den
        c = rng.standard_normal(6)
        f = c[0] + c[1] * u + c[2] * v + c[3] * u * u + c[4] * u * v + c[5] * v * v
        f = np.where(xs @ g > 0.5, f, 0.0)
        got = B.remesh(x, off, nb, xs, f, points=[k])[0]
        if abs(got - c[0]) > 1e-11 * np.abs(c).max():
            return False
    return True


def _pin_stencil():
    x, off, nb, xs, _, _, _ = moved(3, steps=10)
    deg = np.diff(off)
    Q = B.remesh_members(x, off, nb, xs)
    cell = np.argmin(((xs[:, None, :] - x[None, :, :]) ** 2).sum(-1), axis=1)
    for k in (0, 7, 100, 331, 641):
        S = B.ring_stencil(off, nb, k, 2)
        if len(S) != (16 if deg[k] == 5 else 19):
            return False
        if sorted(Q[k]) != sorted(int(p) for p in np.nonzero(np.isin(cell, S))[0]):
            return False
    return True


def _remesh_errors(levels=(3, 4, 5)):
    errs = []
    for lev in levels:
        x, off, nb, xs, _, _, _ = moved(lev)
        F = I.rossby_haurwitz_vorticity
        got = B.remesh(x, off, nb, xs, F(xs))
        errs.append(np.abs(got - F(x)).max())
    return errs


def _pin_third_order():
    e = _remesh_errors()
    return all(e[i] / e[i + 1] > 6.0 for i in range(len(e) - 1))


def _rh_remeshed(level, steps=10):
    x, z, A, off, nb = I.workload_bve(level, with_adjacency=True)
    zc = z.copy()
    for _ in range(steps):
        zc = B.remeshed_step(x, off, nb, zc, A, I.BVE_DT, OMEGA)
    return B.vorticity_error(zc, z, A)


def _pin_rh_remeshed():
    e3, e4 = _rh_remeshed(3), _rh_remeshed(4)
    return e4 < 0.012 and e3 / e4 > 6.0


def test_quadratics_reproduced_exactly():
    assert _pin_quadratic_exact()


def test_stencil_and_cells():
    assert _pin_stencil()


def test_remeshing_error_third_order():
    e = _remesh_errors()
    print("\nmax remeshing error of zeta_RH, levels 3, 4, 5:", e)
    assert all(e[i] / e[i + 1] > 6.0 for i in range(len(e) - 1))


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5])
def test_icosahedral_triangulation_is_delaunay(level):
    from scipy.spatial import ConvexHull
    v, f = I.icosahedral_triangulation(level)
    hull = ConvexHull(v)
    assert sorted(map(tuple, np.sort(f, 1))) == sorted(map(tuple, np.sort(hull.simplices, 1)))


def test_rh_wave_with_remeshing_converges():
    e3, e4 = _rh_remeshed(3), _rh_remeshed(4)
    print(f"\nE_zeta(0.1 day) with remeshing: level 3 {e3:.3e}, level 4 {e4:.3e}")
    assert e4 < 0.012 and e3 / e4 > 6.0


def test_grid_adjacency():
    v, f = I.icosahedral_triangulation(2)
    off, nb = I.grid_adjacency(f, len(v))
    deg = np.diff(off)
    assert (deg == 5).sum() == 12 and (deg == 6).sum() == len(v) - 12
    for k in range(len(v)):
        row = nb[off[k]:off[k + 1]]
        assert list(row) == sorted(row) and k not in row
        for j in row:
            assert k in nb[off[j]:off[j + 1]]


REMESH_MUTATIONS = {6: "orthographic coordinates", 7: "one-ring stencil",
                    8: "starting grid point as the cell", 9: "u v term dropped",
                    10: "weights dropped"}


@pytest.mark.parametrize("m", sorted(REMESH_MUTATIONS))
def test_planted_remesh_mistake_fails_a_pin(m):
    B.set_mutation(m)
    try:
        caught = not (_pin_quadratic_exact() and _pin_stencil() and _pin_third_order()
                      and _pin_rh_remeshed())
    finally:
        B.set_mutation(0)
    assert caught, REMESH_MUTATIONS[m]
