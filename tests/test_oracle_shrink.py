"""Pins of the oracle's shrunk cells (Sec. 3: for nonuniform particles the
clusters are shrunk to bound their particles tightly).

What fixes the answer: with K = 1 every interaction is exact whatever the
boxes, so the CSFMM returns sum_{j != i} w_j; every point lies inside its
leaf's box (local coordinates in [-1, 1]); at high degree on a tiny clustered
set the CSFMM equals the direct sum; without shrinking nothing changes; and,
the reason the paper gives for shrinking, on clustered points the same degree
and MAC need fewer direct pairs and kernel evaluations (the error still
converges with the degree; at a fixed degree its worst case grows, because
the separation test r_t + r_s < MAC R then admits a large cluster next to a
nearly point-like one).
"""
import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I


def clustered(n, seed, spread=0.15):
    """n points in a few tight caps (a strongly nonuniform set)."""
    rng = np.random.default_rng(seed)
    centres = I.random_sphere_points(5, seed + 1)
    c = centres[rng.integers(0, 5, n)]
    v = rng.standard_normal((n, 3))
    v -= np.sum(v * c, axis=1, keepdims=True) * c
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    th = spread * np.abs(rng.standard_normal(n)) * rng.random(n)
    return np.cos(th)[:, None] * c + np.sin(th)[:, None] * v


def _pin_inside():
    pts = clustered(3000, 3)
    u, v, leaf = O.FMM(pts, 4, 0.7, 20, shrink=True).local_coords()
    return np.abs(u).max() <= 1 + 1e-12 and np.abs(v).max() <= 1 + 1e-12


def _pin_high_degree():
    pts = clustered(600, 5)
    w = np.random.default_rng(6).standard_normal(len(pts))
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    fs = O.FMM(pts, 16, 0.5, 12, shrink=True).evaluate(O.KERNEL_LAPLACE, w)[0, :, 0]
    return np.linalg.norm(fs - ds) / np.linalg.norm(ds) < 1e-11


def test_constant_kernel_covers_every_source_once():
    for pts in (clustered(2500, 7), I.random_sphere_points(2000, 8)):
        w = np.random.default_rng(9).standard_normal(len(pts))
        out = O.FMM(pts, 3, 0.7, 12, shrink=True).evaluate(O.KERNEL_ONE, w)[0, :, 0]
        assert np.abs(out - (w.sum() - w)).max() < 1e-11


def test_points_inside_their_boxes():
    assert _pin_inside()


def test_high_degree_equals_direct():
    assert _pin_high_degree()


def test_unshrunk_plan_unchanged_by_the_option():
    pts = I.random_sphere_points(1500, 10)
    w = np.random.default_rng(11).standard_normal(len(pts))
    a = O.FMM(pts, 5, 0.7, 20).evaluate(O.KERNEL_NEWTON, w)
    b = O.FMM(pts, 5, 0.7, 20, shrink=False).evaluate(O.KERNEL_NEWTON, w)
    assert np.array_equal(a, b)


def test_shrinking_cuts_work_on_clustered_points():
    """Shrunk boxes pass the separation test sooner: on clustered points the
    same degree and MAC need fewer direct (PP) pairs and fewer kernel
    evaluations, and the error still converges with the degree."""
    pts = clustered(6000, 12)
    w = np.random.default_rng(13).random(len(pts)) / len(pts)
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)
    info = {}
    for sh in (False, True):
        info[sh] = O.FMM(pts, 6, 0.7, 40, shrink=sh).info()
    print(f"\nPP pairs {info[False]['nPP']} -> {info[True]['nPP']}, "
          f"evaluations {info[False]['evals']} -> {info[True]['evals']}")
    assert info[True]["nPP"] < 0.8 * info[False]["nPP"]
    assert info[True]["evals"] < 0.95 * info[False]["evals"]
    errs = []
    for n in (4, 8, 12):
        fs = O.FMM(pts, n, 0.7, 40, shrink=True).evaluate(O.KERNEL_LAPLACE, w)
        errs.append(np.linalg.norm(fs - ds) / np.linalg.norm(ds))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-9


def test_planted_mistake_box_edge_fails_a_pin():
    O.set_mutation(15)
    try:
        caught = not (_pin_inside() and _pin_high_degree())
    finally:
        O.set_mutation(0)
    assert caught
