"""Plant numbered mistakes in the oracle (on the CPU) and check that the pins
catch each one: a dropped term, a wrong sign, a transposed or wrong index, a
wrong weight, a skipped pass.  This is what makes the pins trustworthy."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I


def _pin_constant_kernel():
    pts = I.random_sphere_points(2000, 5)
    w = np.random.default_rng(6).standard_normal(2000)
    out = O.FMM(pts, 3, 0.7, 12).evaluate(O.KERNEL_ONE, w)[0, :, 0]
    return np.max(np.abs(out - (w.sum() - w))) < 1e-12


def _pin_high_degree_vs_direct():
    pts, A = I.cubed_sphere_grid(16)
    w = I.real_sph_harm(4, 3, pts) * A
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    fs = O.FMM(pts, 14, 0.7, 16).evaluate(O.KERNEL_LAPLACE, w)[0, :, 0]
    return O.rel_l2(fs, ds, A) < 1e-12


def _pin_funk_hecke():
    pts, A, w, ex = I.workload_poisson_y43(16)
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    return O.rel_l2(ds, ex[0], A) < 0.15


def _pin_coverage():
    pts = I.random_sphere_points(1500, 2)
    return O.FMM(pts, 4, 0.7, 10).info()["pairs_covered"] == 1500 ** 2


def _pin_lagrange():
    for n in (2, 5):
        s = O.cheb_nodes(n)
        if not np.allclose(s, np.cos(np.arange(n + 1) * np.pi / n)):
            return False
        c = np.arange(1.0, n + 2)
        for u in (-0.3, 0.77):
            if abs(O.lagrange(n, u) @ np.polyval(c, s) - np.polyval(c, u)) > 1e-12:
                return False
    return True


def _pin_moments():
    pts, A = I.cubed_sphere_grid(16)
    n = 3
    w = np.random.default_rng(1).standard_normal(len(pts))
    f = O.FMM(pts, n, 0.7, 12)
    C = f.cells()
    wb = f.upward(w)[:, 0, :]
    s = O.cheb_nodes(n)
    xs, ws = pts[f.order()], w[f.order()]
    for c in range(len(C["face"])):
        face = C["face"][c]
        ax = face // 2
        a = xs[:, (ax + 1) % 3] / np.abs(xs[:, ax])
        h = (math.pi / 2) / 2 ** (C["level"][c] + 1)
        u = (np.arctan(a) - ((2 * C["ia"][c] + 1) * h - math.pi / 4)) / h
        seg = slice(C["begin"][c], C["end"][c])
        lhs = np.sum(wb[c].reshape(n + 1, n + 1) * (s[:, None] * np.ones(n + 1)[None, :]))
        rhs = np.sum(ws[seg] * u[seg])
        if abs(lhs - rhs) > 1e-11 * (1 + np.abs(ws[seg]).sum()):
            return False
    return True


def _pin_cstc_constant_kernel():
    pts = I.random_sphere_points(2000, 5)
    w = np.random.default_rng(6).standard_normal(2000)
    out = O.FMM(pts, 3, 0.7, 12).evaluate_cstc(O.KERNEL_ONE, w)[0, :, 0]
    return np.max(np.abs(out - (w.sum() - w))) < 1e-12


def _pin_cstc_high_degree_vs_direct():
    pts, A = I.cubed_sphere_grid(8)
    w = I.real_sph_harm(4, 3, pts) * A
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    cs = O.FMM(pts, 14, 0.5, 16).evaluate_cstc(O.KERNEL_LAPLACE, w)[0, :, 0]
    return O.rel_l2(cs, ds, A) < 1e-11


def _pin_biharmonic_eigenvalue():
    pts, A = I.cubed_sphere_grid(32)
    y = I.real_sph_harm(1, 0, pts)
    ds = O.direct(pts, O.KERNEL_BIHARMONIC, y * A)[0, :, 0]
    return O.rel_l2(ds, y / 4.0, A) < 2e-3 and abs(O.dilog(0.5) - 0.5822405264650125) < 1e-15


PINS = [_pin_biharmonic_eigenvalue, _pin_constant_kernel, _pin_high_degree_vs_direct, _pin_funk_hecke,
        _pin_coverage, _pin_lagrange, _pin_moments, _pin_cstc_constant_kernel,
        _pin_cstc_high_degree_vs_direct]

MUTATIONS = {
    1: "PC term dropped",
    2: "Laplace kernel sign flipped",
    3: "M2M uses the wrong child half in xi",
    4: "Chebyshev points cos(k pi/(n+1))",
    5: "PP keeps the i = j term",
    6: "L2P interpolates with u in both directions (transposed operand)",
    7: "MAC comparison reversed",
    8: "barycentric end weights not halved",
    9: "deepest L2L level skipped",
    10: "P2M reads weights by input index instead of sorted position",
    11: "CSTC separation test reversed",
    12: "CSTC drops a leaf that is not well separated",
    13: "CSTC visits the first child twice instead of the fourth",
    14: "dilogarithm reflection drops the log(x) log(1 - x) term",
}


def test_pins_pass_on_the_unmutated_oracle():
    O.set_mutation(0)
    assert all(p() for p in PINS)


@pytest.mark.parametrize("mut", sorted(MUTATIONS))
def test_each_planted_mistake_fails_a_pin(mut):
    try:
        O.set_mutation(mut)
        with np.errstate(all="ignore"):
            failed = [p.__name__ for p in PINS if not p()]
    finally:
        O.set_mutation(0)
    assert failed, f"mutation {mut} ({MUTATIONS[mut]}) passed every pin"
