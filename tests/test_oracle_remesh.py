"""Pins of the oracle's remeshing (Sec. 12: remeshing at every step by local
interpolation; the reading -- a weighted quadratic least-squares fit in
scaled gnomonic coordinates over the particles of a data disc whose weights
vanish smoothly at its edge -- is stated in oracle/bve.py).

What fixes the answer without the oracle: a quadratic in the gnomonic
coordinates of g_k is reproduced exactly at g_k whatever the particles'
positions; a particle that crosses the edge of a data disc changes nothing
discontinuously; the remeshing error of a smooth field falls third-order
with the grid spacing; several fields remeshed together equal each remeshed
alone; the icosahedral triangulation is the Delaunay triangulation (convex
hull) of its vertices, which the GPU's nearest-point walk needs; and with
remeshing the RH wave's E_zeta keeps falling with N as Sec. 12 reports, the
tracer q = z keeps zero mass, and a tracer equal to the absolute vorticity
stays equal to it.  Planted mistakes 6-9 each fail one of these.
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


def _pin_continuous():
    """Move one particle from just inside to just outside the data disc of a
    grid point: the value there moves by ~ the weight at the edge (~1e-12),
    not by a jump."""
    x, off, nb, xs, zs, _, _ = moved(3, steps=3)
    h = B.neighbour_scale(x, off, nb)
    k = 100
    g = x[k]
    e1, e2 = B.tangent_basis(g)
    d = xs @ g
    s = np.hypot(xs @ e1, xs @ e2) / (d * h[k])
    p = int(np.argmin(np.abs(s - B.S_C) + (d <= 0)))
    vals = []
    for target in (B.S_C * (1 - 1e-4), B.S_C * (1 + 1e-4)):
        y = xs.copy()
        t = y[p] - (y[p] @ g) * g
        t /= np.linalg.norm(t)
        ang = np.arctan(target * h[k])
        y[p] = np.cos(ang) * g + np.sin(ang) * t
        vals.append(B.remesh(x, off, nb, y, zs, points=[k])[0])
    return abs(vals[1] - vals[0]) < 1e-9 * np.abs(zs).max()


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
    return e4 < 0.01 and e3 / e4 > 6.0


def test_quadratics_reproduced_exactly():
    assert _pin_quadratic_exact()


def test_remeshing_continuous_in_positions():
    assert _pin_continuous()


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
    assert e4 < 0.01 and e3 / e4 > 6.0


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


def test_fields_share_the_fit():
    """Remeshing several fields at once equals remeshing each alone (one
    normal matrix, one right-hand side per field)."""
    x, off, nb, xs, zs, _, _ = moved(3, steps=5)
    q = np.sin(3 * xs[:, 0]) + xs[:, 2]
    both = B.remesh(x, off, nb, xs, np.stack([zs, q]))
    assert np.allclose(both[0], B.remesh(x, off, nb, xs, zs), rtol=0, atol=1e-13)
    assert np.allclose(both[1], B.remesh(x, off, nb, xs, q), rtol=0, atol=1e-13)


def test_tracer_mass_vanishes_and_absolute_vorticity_tracer():
    """Sec. 12: the tracer q = z has zero mass by symmetry, which the symmetric
    icosahedral grid keeps to rounding; a tracer initialised to the absolute
    vorticity zeta + 2 Omega z is carried like it (Eq. BVE), so after remeshed
    steps it equals the remeshed zeta + 2 Omega z at the grid points up to the
    remeshing error of z."""
    x, z, A, off, nb = I.workload_bve(3, with_adjacency=True)
    q = x[:, 2].copy()
    qa = z + 2 * OMEGA * x[:, 2]
    zc = z.copy()
    for _ in range(5):
        xs, zs = B.rk4_step(x, zc, A, I.BVE_DT, OMEGA)
        zc, q, qa = B.remesh(x, off, nb, xs, np.stack([zs, q, qa]))
    m, qmax = B.tracer_properties(q, A)
    assert abs(m) < 1e-13 and qmax <= 1.0 + 1e-3
    gap = np.abs(qa - (zc + 2 * OMEGA * x[:, 2])).max()
    print(f"\nabsolute-vorticity tracer gap {gap / np.abs(zc).max():.2e} of max|zeta|")
    assert gap < 4e-3 * np.abs(zc).max()


REMESH_MUTATIONS = {6: "orthographic coordinates", 7: "h_k scaling dropped",
                    8: "u v term dropped", 9: "weights dropped"}


@pytest.mark.parametrize("m", sorted(REMESH_MUTATIONS))
def test_planted_remesh_mistake_fails_a_pin(m):
    B.set_mutation(m)
    try:
        caught = not (_pin_quadratic_exact() and _pin_continuous() and _pin_third_order()
                      and _pin_rh_remeshed())
    finally:
        B.set_mutation(0)
    assert caught, REMESH_MUTATIONS[m]


def test_quadratics_reproduced_on_variable_resolution_grid():
    """Quadratic exactness where h_k varies 4.5x over the sphere (Schmidt-mapped
    icosahedral grid, particles moved by seeded random steps of up to 0.9 of
    the local spacing), at the finest and coarsest grid points and between."""
    v, faces = I.icosahedral_triangulation(3)
    x = I.schmidt_transform(v, 0.5)
    off, nb = I.grid_adjacency(faces, len(x))
    h = B.neighbour_scale(x, off, nb)
    assert h.max() / h.min() > 3.0
    rng = np.random.default_rng(I.MASTER_SEED + 73)
    d = rng.normal(size=x.shape)
    d -= (d * x).sum(1, keepdims=True) * x
    d *= (0.9 * h * rng.uniform(size=len(x)) / np.linalg.norm(d, axis=1))[:, None]
    xs = x + d
    xs /= np.linalg.norm(xs, axis=1, keepdims=True)
    picks = [int(np.argmax(x[:, 2])), int(np.argmin(x[:, 2])), int(np.argmin(h)),
             int(np.argmax(h)), 200, 400]
    for k in picks:
        g = x[k]
        a = np.array([0.3, 0.8, -0.5]) if abs(g[0]) < 0.9 else np.array([0.0, 1.0, 0.2])
        e1 = a - (a @ g) * g
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(g, e1)
        den = (xs @ g) * h[k]
        u, w = (xs @ e1) / den, (xs @ e2) / den
        c = rng.standard_normal(6)
        f = c[0] + c[1] * u + c[2] * w + c[3] * u * u + c[4] * u * w + c[5] * w * w
        f = np.where(xs @ g > 0.5, f, 0.0)
        got = B.remesh(x, off, nb, xs, f, points=[k])[0]
        assert abs(got - c[0]) <= 1e-11 * np.abs(c).max(), k
