"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: they check closed forms
(Funk-Hecke eigenvalues, Sec. 2), printed values (Table "grids"), exactness
properties of interpolation (Sec. 4, Eq. interpolation_identity), integer
identities of the interaction lists (Sec. 8), and invariants (rotation,
linearity, mean), chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them
(test_oracle_mutations.py plants such mistakes).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I
from conftest import golden


# --------------------------------------------------------------------------
# Input grid (Sec. 3 / Table "grids")
# --------------------------------------------------------------------------

def test_grid_sizes_match_table_grids():
    for L, N, dphi in golden("grids_cubed_sphere.txt"):
        m = 2 ** int(L)
        if m > 256:
            assert 6 * m * m == int(N)
            continue
        pts, A = I.cubed_sphere_grid(m)
        assert len(pts) == int(N)
        got = math.sqrt(4 * math.pi / len(pts)) * 180 / math.pi
        assert abs(got - float(dphi)) <= 0.006 * float(dphi)


@pytest.mark.parametrize("m", [8, 32, 64])
def test_grid_areas_sum_to_sphere(m):
    pts, A = I.cubed_sphere_grid(m)
    assert np.allclose(np.linalg.norm(pts, axis=1), 1.0, atol=1e-15)
    assert abs(A.sum() - 4 * math.pi) < 1e-12
    # area ratio smallest/largest about 0.7 (Sec. 3)
    assert 0.6 < A.min() / A.max() < 0.8


def test_real_harmonics_orthonormal():
    pts, A = I.cubed_sphere_grid(64)
    idx = [(0, 0), (1, 0), (1, 1), (2, -1), (4, 3), (5, 4), (8, 5), (8, -5)]
    Y = np.stack([I.real_sph_harm(n, m, pts) for n, m in idx])
    G = (Y * A) @ Y.T
    assert np.max(np.abs(G - np.eye(len(idx)))) < 2e-3
    assert abs(I.real_sph_harm(0, 0, pts)[0] - 1 / (2 * math.sqrt(math.pi))) < 1e-15


def test_real_harmonics_match_scipy():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    pts = I.random_sphere_points(200, 7)
    th = np.arccos(np.clip(pts[:, 2], -1, 1))
    ph = np.arctan2(pts[:, 1], pts[:, 0])
    for n, m in [(4, 3), (8, 5), (3, 0), (6, -2)]:
        Yc = sp.sph_harm_y(n, abs(m), th, ph)
        cs = (-1) ** abs(m)  # scipy includes the Condon-Shortley phase
        if m > 0:
            ref = math.sqrt(2) * cs * Yc.real
        elif m < 0:
            ref = math.sqrt(2) * cs * Yc.imag
        else:
            ref = Yc.real
        assert np.max(np.abs(I.real_sph_harm(n, m, pts) - ref)) < 1e-12


# --------------------------------------------------------------------------
# Direct sum: closed forms (Sec. 2) and convergence (Sec. 10.2)
# --------------------------------------------------------------------------

def _e(a, b, A):
    return O.rel_l2(a, b, A)


def test_laplace_funk_hecke_y43_second_order():
    """int G_L Y_{4,3} = Y_{4,3}/20 (Funk-Hecke; Sec. 2.1), midpoint rule
    error falling ~4x per halving of the spacing (Sec. 10.2)."""
    errs = []
    for m in (16, 32, 64):
        pts, A, w, ex = I.workload_poisson_y43(m)
        ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
        errs.append(_e(ds, ex[0], A))
    assert errs[1] < 0.05
    for a, b in zip(errs, errs[1:]):
        assert 3.0 < a / b < 4.5


def test_laplace_y00_constant():
    """Eq. (G_L_2): int G_L Y_00 = (1 - ln 2)/(2 sqrt(pi))."""
    pts, A = I.cubed_sphere_grid(32)
    y00 = 1 / (2 * math.sqrt(math.pi))
    ds = O.direct(pts, O.KERNEL_LAPLACE, y00 * A)[0, :, 0]
    ref = (1 - math.log(2)) / (2 * math.sqrt(math.pi))
    assert np.max(np.abs(ds - ref)) / ref < 1e-2


def test_newton_funk_hecke_first_order():
    """sum_n P_n = 1/sqrt(2(1-x)) (Eq. Legendre) gives
    int Y_n / sqrt(2(1 - x.y)) = 4 pi/(2n+1) Y_n.  Omitting the singular
    self term makes the midpoint rule first order here."""
    errs = []
    for m in (16, 32, 64):
        pts, A = I.cubed_sphere_grid(m)
        f = I.real_sph_harm(3, 2, pts)
        ds = O.direct(pts, O.KERNEL_NEWTON, f * A)[0, :, 0]
        errs.append(_e(ds, 4 * math.pi / 7 * f, A))
    assert errs[2] < 0.06
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.3


def test_biot_savart_rh_wave_velocity():
    """K_BS = grad_x G_L x x (Sec. 2.3), so the Biot-Savart sum of the RH
    vorticity approximates grad_S psi x x with psi = int G_L zeta."""
    errs = []
    for m in (16, 32, 64):
        pts, A = I.cubed_sphere_grid(m)
        z = I.rossby_haurwitz_vorticity(pts)
        u = O.direct(pts, O.KERNEL_BIOT_SAVART, z * A)[0]
        errs.append(_e(u, I.rossby_haurwitz_velocity(pts), A))
    assert errs[1] < 0.01
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.5


def test_direct_rotation_invariance():
    pts = I.random_sphere_points(600, 11)
    Rm = I.random_rotation(12)
    w = np.random.default_rng(13).standard_normal(600)
    for k in (O.KERNEL_LAPLACE, O.KERNEL_NEWTON):
        a = O.direct(pts, k, w)[0, :, 0]
        b = O.direct(pts @ Rm.T, k, w)[0, :, 0]
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
    a = O.direct(pts, O.KERNEL_BIOT_SAVART, w)[0]
    b = O.direct(pts @ Rm.T, O.KERNEL_BIOT_SAVART, w)[0]
    assert np.max(np.abs(a @ Rm.T - b)) <= 1e-12 * np.max(np.abs(a))


def test_direct_zero_mean_and_linearity():
    pts, A = I.cubed_sphere_grid(32)
    f = I.real_sph_harm(2, 1, pts) + 0.5 * I.real_sph_harm(3, -3, pts)
    w = np.stack([f * A, 2.0 * f * A, A * I.real_sph_harm(1, 0, pts)])
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[:, :, 0]
    assert abs(np.sum(ds[0] * A)) < 1e-4 * np.sqrt(np.sum(ds[0] ** 2 * A))
    assert np.max(np.abs(ds[1] - 2 * ds[0])) < 1e-14 * np.max(np.abs(ds[1]))


def test_direct_omits_only_self_term():
    """With K = 1 the sum is sum_{j != i} w_j exactly."""
    w = np.random.default_rng(3).standard_normal(257)
    pts = I.random_sphere_points(257, 4)
    ds = O.direct(pts, O.KERNEL_ONE, w)[0, :, 0]
    assert np.max(np.abs(ds - (w.sum() - w))) < 1e-13


# --------------------------------------------------------------------------
# Barycentric interpolation (Sec. 4)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 6, 12])
def test_lagrange_basis_properties(n):
    s = O.cheb_nodes(n)
    assert np.allclose(s, np.cos(np.arange(n + 1) * np.pi / n), atol=0, rtol=0)
    for j in range(n + 1):
        assert np.array_equal(O.lagrange(n, s[j]), np.eye(n + 1)[j])
    rng = np.random.default_rng(n)
    c = rng.standard_normal(n + 1)
    for u in rng.uniform(-1, 1, 20):
        L = O.lagrange(n, u)
        assert abs(L.sum() - 1) < 1e-13
        # exact for polynomials of degree <= n (numpy's polyval as reference)
        assert abs(L @ np.polyval(c, s) - np.polyval(c, u)) < 1e-12


def test_lagrange_matches_scipy_barycentric():
    interp = pytest.importorskip("scipy.interpolate")
    n = 9
    s = O.cheb_nodes(n)
    f = np.exp(np.sin(3 * s))
    bi = interp.BarycentricInterpolator(s, f)
    for u in np.linspace(-0.99, 0.99, 17):
        assert abs(O.lagrange(n, u) @ f - bi(u)) < 1e-13


# --------------------------------------------------------------------------
# Tree (Sec. 3) and interaction lists (Sec. 8)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m,n,N0,shape", [
    (32, 8, 64, (126, 96, 3)),       # 6144 points: leaves at level 2, 64 points each
    (256, 10, 400, (2046, 1536, 5)),  # 393,216 points: leaves at level 4
    (64, 3, 36, (2046, 1536, 5)),    # 24,576 points: 16 per leaf at level 4
    (16, 2, 64, (30, 24, 2)),         # 1,536 points: 64 per leaf at level 1
])
def test_tree_shape_uniform_grid(m, n, N0, shape):
    pts, A = I.cubed_sphere_grid(m)
    f = O.FMM(pts, n, 0.7, N0)
    info = f.info()
    assert (info["ncells"], info["nleaves"], info["nlevels"]) == shape
    C = f.cells()
    leaf = C["child"].max(axis=1) < 0
    cnt = C["end"] - C["begin"]
    assert np.all(cnt[leaf] <= N0) and np.all(cnt[~leaf] > N0)
    assert cnt[C["level"] == 0].sum() == len(pts)
    # leaves partition the sorted points
    lb = np.sort(C["begin"][leaf])
    le = np.sort(C["end"][leaf])
    assert lb[0] == 0 and le[-1] == len(pts) and np.array_equal(lb[1:], le[:-1])
    assert np.array_equal(np.sort(f.order()), np.arange(len(pts)))


def test_tree_cells_bound_their_points():
    pts = I.random_sphere_points(5000, 21)
    f = O.FMM(pts, 4, 0.7, 30)
    C = f.cells()
    xs = pts[f.order()]
    assert np.allclose(np.linalg.norm(C["centre"], axis=1), 1.0, atol=1e-15)
    for c in range(len(C["face"])):
        seg = xs[C["begin"][c]:C["end"][c]]
        d = np.linalg.norm(seg - C["centre"][c], axis=1)
        assert np.all(d <= C["radius"][c] * (1 + 1e-12))
    u, v, leaf = f.local_coords()
    assert np.all(np.abs(u) <= 1 + 1e-12) and np.all(np.abs(v) <= 1 + 1e-12)


@pytest.mark.parametrize("seed,N,n,N0,theta", [(1, 3000, 4, 20, 0.7), (2, 6144, 6, 40, 0.5),
                                                (3, 800, 2, 5, 0.9)])
def test_lists_cover_every_pair_once(seed, N, n, N0, theta):
    pts = I.random_sphere_points(N, seed)
    f = O.FMM(pts, n, theta, N0)
    info = f.info()
    assert info["pairs_covered"] == N * N
    C = f.cells()
    cnt = C["end"] - C["begin"]
    L = f.lists()
    # exact membership count per (target point, source point) on a sample
    cover = np.zeros((N, N), dtype=np.int32) if N <= 3000 else None
    leaf = C["child"].max(axis=1) < 0
    for ty, (t, s) in L.items():
        if ty == O.PP:
            assert np.all(leaf[t]) and np.all(leaf[s])
        if ty == O.PC:
            assert np.all(leaf[t]) and np.all(~leaf[s])
        if ty == O.CP:
            assert np.all(~leaf[t]) and np.all(leaf[s])
        if ty == O.CC:
            assert np.all(~leaf[t]) and np.all(~leaf[s])
        if ty != O.PP:
            R = np.linalg.norm(C["centre"][t] - C["centre"][s], axis=1)
            assert np.all(C["radius"][t] + C["radius"][s] < theta * R)
        if cover is not None:
            for a, b in zip(t, s):
                cover[C["begin"][a]:C["end"][a], C["begin"][b]:C["end"][b]] += 1
    if cover is not None:
        assert np.all(cover == 1)


def test_fmm_constant_kernel_is_exact():
    """With K = 1 every interpolation is exact (partition of unity), so the
    FMM equals sum_{j != i} w_j to rounding."""
    pts = I.random_sphere_points(4000, 5)
    w = np.random.default_rng(6).standard_normal((2, 4000))
    f = O.FMM(pts, 3, 0.7, 12)
    out = f.evaluate(O.KERNEL_ONE, w)[:, :, 0]
    ref = w.sum(axis=1, keepdims=True) - w
    assert np.max(np.abs(out - ref)) < 1e-12


def _cell_local(pts, C, c):
    """Local (u, v) of points in the frame of cell c, from the face
    conventions (face axis = largest |component|, a = x_u/|x_axis| ...)."""
    face = C["face"][c]
    ax = face // 2
    u_ax, v_ax = (ax + 1) % 3, (ax + 2) % 3
    a = pts[:, u_ax] / np.abs(pts[:, ax])
    b = pts[:, v_ax] / np.abs(pts[:, ax])
    h = (math.pi / 2) / 2 ** (C["level"][c] + 1)
    xm = (2 * C["ia"][c] + 1) * h - math.pi / 4
    ym = (2 * C["ib"][c] + 1) * h - math.pi / 4
    return (np.arctan(a) - xm) / h, (np.arctan(b) - ym) / h


@pytest.mark.parametrize("n", [3, 6])
def test_upward_pass_moment_identity(n):
    """Sum_k wbar_k p(s_k) = sum_j w_j p(y_j) for every polynomial p of degree
    <= n in each variable of the cell's local coordinates, after P2M and after
    every M2M level (Eqs. PC, interpolation_identity, upwardpass2)."""
    pts, A = I.cubed_sphere_grid(32)
    w = np.random.default_rng(n).standard_normal(len(pts))
    f = O.FMM(pts, n, 0.7, 24)
    C = f.cells()
    wb = f.upward(w)[:, 0, :]
    s = O.cheb_nodes(n)
    xs = pts[f.order()]
    ws = w[f.order()]
    rng = np.random.default_rng(99)
    for c in rng.choice(len(C["face"]), 25, replace=False):
        seg = slice(C["begin"][c], C["end"][c])
        u, v = _cell_local(xs[seg], C, c)
        for (da, db) in [(0, 0), (1, 0), (0, 1), (n, n), (n - 1, 2)]:
            lhs = np.sum(wb[c].reshape(n + 1, n + 1) * np.outer(s ** da, s ** db))
            rhs = np.sum(ws[seg] * u ** da * v ** db)
            assert abs(lhs - rhs) < 1e-11 * (1 + np.sum(np.abs(ws[seg])))


# --------------------------------------------------------------------------
# FMM against the direct sum (Sec. 10.3)
# --------------------------------------------------------------------------

def test_fmm_equals_direct_sum_at_high_degree_tiny_n():
    pts, A = I.cubed_sphere_grid(16)
    f_ = I.real_sph_harm(4, 3, pts)
    w = f_ * A
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    fm = O.FMM(pts, 14, 0.7, 16)
    assert fm.info()["nCC"] > 0 and fm.info()["nPC"] > 0
    fs = fm.evaluate(O.KERNEL_LAPLACE, w)[0, :, 0]
    assert O.rel_l2(fs, ds, A) < 1e-12


def test_fmm_error_decreases_with_degree_and_mac():
    pts, A, w, ex = I.workload_poisson_y43(32)
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    errs = {}
    for th in (0.5, 0.7, 0.9):
        for n in (2, 4, 6, 8):
            fs = O.FMM(pts, n, th, 16).evaluate(O.KERNEL_LAPLACE, w)[0, :, 0]
            errs[th, n] = O.rel_l2(fs, ds, A, ex[0])
    for th in (0.5, 0.7, 0.9):
        e = [errs[th, n] for n in (2, 4, 6, 8)]
        assert all(a > b for a, b in zip(e, e[1:])), e
    for n in (2, 4, 6, 8):
        assert errs[0.5, n] < errs[0.7, n] < errs[0.9, n]


def test_fmm_error_magnitude_band_vs_paper_table():
    """Order of magnitude of Table "csfmmerrors" (Y_{4,3}); the paper's grid
    and cluster radius differ, so this is a band, not parity."""
    pts, A, w, ex = I.workload_poisson_y43(128)
    tg = np.sort(np.random.default_rng(1).choice(len(pts), 1000, replace=False))
    ds = O.direct(pts, O.KERNEL_LAPLACE, w, tg)[0, :, 0]
    for mac, n, e_paper in golden("csfmm_errors_y43.txt"):
        mac, n, e_paper = float(mac), int(n), float(e_paper)
        fs = O.FMM(pts, n, mac, 4 * n * n).evaluate(O.KERNEL_LAPLACE, w, tg)[0, :, 0]
        e = O.rel_l2(fs, ds, A[tg], ex[0, tg])
        assert e_paper / 300 < e < e_paper * 3, (mac, n, e, e_paper)


def test_fmm_rotation_consistency():
    pts, A = I.cubed_sphere_grid(32)
    f_ = I.real_sph_harm(4, 3, pts)
    w = f_ * A
    Rm = I.random_rotation(5)
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    a = O.FMM(pts, 5, 0.7, 30).evaluate(O.KERNEL_LAPLACE, w)[0, :, 0]
    b = O.FMM(pts @ Rm.T, 5, 0.7, 30).evaluate(O.KERNEL_LAPLACE, w)[0, :, 0]
    ea, eb = O.rel_l2(a, ds, A), O.rel_l2(b, ds, A)
    assert O.rel_l2(a, b, A, ds) <= ea + eb
    assert 0.1 < ea / eb < 10


def test_fmm_biot_savart_and_targets_subset():
    pts, A, w, ex = I.workload_rh_biot_savart(32)
    ds = O.direct(pts, O.KERNEL_BIOT_SAVART, w)[0]
    fm = O.FMM(pts, 8, 0.7, 40)
    fs = fm.evaluate(O.KERNEL_BIOT_SAVART, w)[0]
    assert O.rel_l2(fs, ds, A) < 1e-6
    tg = np.array([0, 17, 4000, 6143, 17])
    sub = fm.evaluate(O.KERNEL_BIOT_SAVART, w, tg)[0]
    assert np.array_equal(sub, fs[tg])


def test_fmm_linearity_multi_rhs():
    pts, A = I.cubed_sphere_grid(16)
    rng = np.random.default_rng(8)
    w = rng.standard_normal((3, len(pts)))
    w[2] = 2 * w[0] - 3 * w[1]
    out = O.FMM(pts, 4, 0.7, 20).evaluate(O.KERNEL_NEWTON, w)[:, :, 0]
    assert np.max(np.abs(out[2] - (2 * out[0] - 3 * out[1]))) < 1e-12 * np.max(np.abs(out))
