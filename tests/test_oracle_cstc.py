"""Pins of the oracle's cubed sphere tree code (Sec. 7, Algorithm "CSTC").

The paper prints no CSTC errors, so the CSTC oracle is pinned by what the
mathematics fixes: with K = 1 every proxy interaction is exact (partition of
unity), so the result is sum_{j != i} w_j exactly iff every source is covered
once per target; at high degree on a tiny grid it equals the direct sum; its
error falls with the degree and grows with the MAC; it approximates the same
closed form (Funk-Hecke) as the direct sum; and it agrees with the CSFMM on
the same tree to within their truncation errors.
"""
import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I


def clustered_points(n, seed):
    """n points in a spherical cap of angular radius 0.3 around (1, 1, 1)/sqrt(3)
    plus n/4 uniform points: a ragged, non-uniform tree."""
    rng = np.random.default_rng(seed)
    c = np.ones(3) / np.sqrt(3.0)
    v = rng.standard_normal((n, 3))
    v -= np.outer(v @ c, c)
    v /= np.linalg.norm(v, axis=1)[:, None]
    th = 0.3 * np.sqrt(rng.random(n))
    cap = np.cos(th)[:, None] * c + np.sin(th)[:, None] * v
    return np.vstack([cap, I.random_sphere_points(n // 4, seed + 1)])


POINT_SETS = [
    ("cubed m=16", lambda: I.cubed_sphere_grid(16)[0], 4, 0.7, 30),
    ("random 3000", lambda: I.random_sphere_points(3000, 7), 5, 0.7, 20),
    ("clustered cap 2000 + 500", lambda: clustered_points(2000, 3), 3, 0.8, 12),
    ("random 800, N0 = 1", lambda: I.random_sphere_points(800, 9), 2, 0.9, 1),
]


@pytest.mark.parametrize("name,mk,n,theta,N0", POINT_SETS)
def test_cstc_constant_kernel_covers_every_source_once(name, mk, n, theta, N0):
    pts = mk()
    w = np.random.default_rng(4).standard_normal(len(pts))
    out, st = O.FMM(pts, n, theta, N0).evaluate_cstc(O.KERNEL_ONE, w, with_stats=True)
    ref = w.sum() - w
    assert np.max(np.abs(out[0, :, 0] - ref)) <= 1e-12 * np.abs(w).sum(), name
    assert st["pc"] > 0 and st["pp"] > 0


def test_cstc_equals_direct_sum_at_high_degree_tiny_n():
    pts, A = I.cubed_sphere_grid(8)
    w = I.real_sph_harm(4, 3, pts) * A
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    cs = O.FMM(pts, 14, 0.5, 16).evaluate_cstc(O.KERNEL_LAPLACE, w)[0, :, 0]
    assert O.rel_l2(cs, ds, A) < 1e-11


def test_cstc_error_decreases_with_degree_and_grows_with_mac():
    pts, A, w, ex = I.workload_poisson_y43(32)
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    e_n = [O.rel_l2(O.FMM(pts, n, 0.7, 64).evaluate_cstc(O.KERNEL_LAPLACE, w)[0, :, 0], ds, A)
           for n in (2, 4, 6, 8)]
    assert all(a > 4 * b for a, b in zip(e_n, e_n[1:])), e_n
    e_t = [O.rel_l2(O.FMM(pts, 4, t, 64).evaluate_cstc(O.KERNEL_LAPLACE, w)[0, :, 0], ds, A)
           for t in (0.5, 0.7, 0.9)]
    assert e_t[0] < e_t[1] < e_t[2], e_t


def test_cstc_approximates_the_funk_hecke_closed_form():
    """int G_L(x, y) Y43(y) dS(y) = -Y43(x)/20: the CSTC at n = 8 reaches the
    same distance from the closed form as the direct sum (quadrature error)."""
    pts, A, w, ex = I.workload_poisson_y43(32)
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    cs = O.FMM(pts, 8, 0.7, 64).evaluate_cstc(O.KERNEL_LAPLACE, w)[0, :, 0]
    e_ds = O.rel_l2(ds, ex[0], A)
    e_cs = O.rel_l2(cs, ex[0], A)
    assert e_ds < 0.05  # second-order quadrature error at m = 32
    assert abs(e_cs - e_ds) < 1e-3 * e_ds


@pytest.mark.parametrize("kernel", [O.KERNEL_NEWTON, O.KERNEL_BIOT_SAVART, O.KERNEL_LAPLACE])
def test_cstc_converges_to_direct_sum_for_each_kernel(kernel):
    """E(CSTC, DS) falls by > 5x per two degrees for every kernel, and the
    particle-cluster separation test r_s < MAC R (looser than the CSFMM's
    r_t + r_s < MAC R at the same MAC) leaves it above the CSFMM's error."""
    pts, A = I.cubed_sphere_grid(32)
    w = I.land_mask_field(pts, 12) * A
    ds = O.direct(pts, kernel, w)[0]
    e_cs, e_fm = [], []
    for n in (4, 6, 8):
        f = O.FMM(pts, n, 0.7, 64)
        e_cs.append(O.rel_l2(f.evaluate_cstc(kernel, w)[0], ds))
        e_fm.append(O.rel_l2(f.evaluate(kernel, w)[0], ds))
    assert all(a > 5 * b for a, b in zip(e_cs, e_cs[1:])), e_cs
    assert all(c > f for c, f in zip(e_cs, e_fm)), (e_cs, e_fm)
    assert e_cs[-1] < 1e-5


def test_cstc_targets_subset_and_multi_rhs():
    pts = I.random_sphere_points(2500, 11)
    rng = np.random.default_rng(2)
    W = rng.standard_normal((3, len(pts)))
    f = O.FMM(pts, 5, 0.7, 20)
    full = f.evaluate_cstc(O.KERNEL_LAPLACE, W)
    tg = np.array([0, 17, 2499, 1200, 17])
    sub = f.evaluate_cstc(O.KERNEL_LAPLACE, W, targets=tg)
    assert np.array_equal(sub, full[:, tg])
    for r in range(3):
        one = f.evaluate_cstc(O.KERNEL_LAPLACE, W[r])
        assert np.array_equal(one[0], full[r])
    lin = f.evaluate_cstc(O.KERNEL_LAPLACE, 2.0 * W[0] - W[1])[0]
    assert np.max(np.abs(lin - (2.0 * full[0] - full[1]))) < 1e-12 * np.abs(full[:2]).max()
