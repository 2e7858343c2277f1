"""GPU parity of shrunk cells (plan option shrink; Sec. 3) through the C ABI
against the oracle's shrunk tree on the same seeded inputs.

Bars: the same boxes, centres and radii bit for bit and the same interaction
lists; FP64 CSFMM and CSTC relative l2 <= 1e-12 against the oracle; FP32 bulk
against the oracle direct sum at most the per-case bar of fp32_bars.py (about
4x the error measured on GB300); K = 1 exact.
"""
import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I
from gpu_util import cuda_or_skip, dev, cell_keys
from fp32_bars import check as check32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def C():
    from paper_2508_13550_gb300 import csfmm
    return csfmm


def clustered(n, seed, spread=0.15):
    rng = np.random.default_rng(seed)
    centres = I.random_sphere_points(5, seed + 1)
    c = centres[rng.integers(0, 5, n)]
    v = rng.standard_normal((n, 3))
    v -= np.sum(v * c, axis=1, keepdims=True) * c
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    th = spread * np.abs(rng.standard_normal(n)) * rng.random(n)
    return np.cos(th)[:, None] * c + np.sin(th)[:, None] * v


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


SETS = [
    ("clustered 6000 n=6 N0=40", lambda: clustered(6000, 12), 6, 0.7, 40),
    ("random 5000 n=5 N0=30 MAC 0.5", lambda: I.random_sphere_points(5000, 14), 5, 0.5, 30),
    ("icosahedral L4 n=4 N0=16", lambda: I.icosahedral_grid(4)[0], 4, 0.8, 16),
    ("clustered 800, N0=1", lambda: clustered(800, 15, 0.05), 3, 0.7, 1),
]


@pytest.mark.parametrize("name,mk,n,theta,N0", SETS)
def test_tree_and_lists_identical(torch, C, name, mk, n, theta, N0):
    pts = mk()
    ref = O.FMM(pts, n, theta, N0, shrink=True)
    P = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, n, theta, N0, shrink=True)
    st, info = C.plan_stats(P), ref.info()
    assert (st["ncells"], st["nleaves"]) == (info["ncells"], info["nleaves"])
    g, o = C.plan_export_cells(P), ref.cells()
    gk, ok = cell_keys(g), cell_keys(o)
    gi = {k: i for i, k in enumerate(gk)}
    perm = np.array([gi[k] for k in ok])
    assert np.array_equal(g["centre"][perm], o["centre"])
    assert np.array_equal(g["radius"][perm], o["radius"])
    inv = np.empty(len(perm), dtype=np.int64)
    inv[perm] = np.arange(len(perm))
    for ty, (t_o, s_o) in ref.lists().items():
        t_g, s_g = C.plan_export_list(P, ty)
        assert sorted(zip(t_o.tolist(), s_o.tolist())) == sorted(
            zip(inv[t_g].tolist(), inv[s_g].tolist())), ty
    assert sum(st["evals"]) == info["evals"]


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("name,mk,n,theta,N0", SETS)
def test_fp64_matches_oracle(torch, C, name, mk, n, theta, N0, kernel):
    pts = mk()
    W = np.random.default_rng(16).standard_normal((2, len(pts))) / len(pts)
    ref = O.FMM(pts, n, theta, N0, shrink=True).evaluate(kernel, W)
    P = C.plan_create(dev(torch, pts), kernel, n, theta, N0, shrink=True)
    got = C.evaluate(P, dev(torch, W)).cpu().numpy()
    assert rel(got, ref) < 1e-12, (name, kernel, rel(got, ref))


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_fp32_bulk_and_cstc(torch, C, kernel):
    pts = clustered(20000, 17)
    w = np.random.default_rng(18).random(len(pts)) / len(pts)
    tg = np.sort(np.random.default_rng(19).choice(len(pts), 500, replace=False))
    ds = O.direct(pts, kernel, w, tg)
    P = C.plan_create(dev(torch, pts), kernel, 10, 0.5, 100, precision=C.FP32_BULK, shrink=True)
    got = C.evaluate(P, dev(torch, np.atleast_2d(w))).cpu().numpy()[:, tg]
    print(f"\nkernel {kernel} FP32 bulk shrunk: {rel(got, ds):.2e}")
    check32(f"fmm32-shrunk-clustered-k{kernel}", rel(got, ds))
    small = clustered(3000, 20)
    ws = np.random.default_rng(21).random(len(small))
    ref = O.FMM(small, 5, 0.7, 20, shrink=True).evaluate_cstc(kernel, ws)
    P64 = C.plan_create(dev(torch, small), kernel, 5, 0.7, 20, shrink=True)
    assert rel(C.evaluate_cstc(P64, dev(torch, np.atleast_2d(ws))).cpu().numpy(), ref) < 1e-12


def test_constant_kernel_and_separate_targets(torch, C):
    src, tgt = clustered(4000, 22), clustered(700, 23)
    w = np.random.default_rng(24).standard_normal(len(src))
    for prec, tol in ((C.FP64, 1e-13), (C.FP32_BULK, 1e-7)):
        P = C.plan_create_targets(dev(torch, src), dev(torch, tgt), C.KERNEL_ONE, 3, 0.7, 16,
                                  precision=prec, shrink=True)
        got = C.evaluate(P, dev(torch, np.atleast_2d(w))).cpu().numpy()[0, :, 0]
        assert np.abs(got - w.sum()).max() < tol * np.abs(w).sum()
    ref = O.fmm_targets(src, tgt, 6, 0.7, 30, O.KERNEL_NEWTON, w, shrink=True)
    P = C.plan_create_targets(dev(torch, src), dev(torch, tgt), C.KERNEL_NEWTON, 6, 0.7, 30,
                              shrink=True)
    assert rel(C.evaluate(P, dev(torch, np.atleast_2d(w))).cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("shrink", [False, True])
def test_variable_resolution_grid_sal(torch, C, shrink):
    """The SAL kernel on a variable-resolution (Schmidt-mapped icosahedral)
    grid, the stand-in for the paper's MPAS SAL runs: FP64 parity with the
    oracle and the FP32-bulk error against the FP64 direct sum."""
    pts, A = I.variable_resolution_grid(5)
    eta = I.land_mask_field(pts, 72) * A  # a sea-surface-height-like field
    ref = O.FMM(pts, 6, 0.7, 40, shrink=shrink).evaluate(O.KERNEL_SAL, eta)
    P = C.plan_create(dev(torch, pts), C.KERNEL_SAL, 6, 0.7, 40, shrink=shrink)
    assert rel(C.evaluate(P, dev(torch, np.atleast_2d(eta))).cpu().numpy(), ref) < 1e-12
    ds = O.direct(pts, O.KERNEL_SAL, eta)
    P32 = C.plan_create(dev(torch, pts), C.KERNEL_SAL, 8, 0.7, 64, precision=C.FP32_BULK,
                        shrink=shrink)
    e32 = rel(C.evaluate(P32, dev(torch, np.atleast_2d(eta))).cpu().numpy(), ds)
    print(f"\nSAL on the variable-resolution grid, shrink={shrink}: FP32 bulk {e32:.2e}")
    check32(f"fmm32-sal-varres-shrink{int(shrink)}", e32)
