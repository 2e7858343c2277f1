"""Symmetric far field of the FP32-bulk form: a CC entry (T, S) whose mirror
(S, T) is also a CC entry is evaluated once, the P x P kernel matrix between
the proxies of T and S serving both cells (Sec. 5, Eq. CC with K(x, y) =
K(y, x)).  The result is compared with the oracle FMM on the same tree,
degree and MAC (so that only the FP32 rounding of the GPU path remains)
within the per-case FP32 bar, and with the direct evaluation of every CC
entry (CSFMM_SCHED_NO_SYMMETRIC) within the FP32 rounding of the two."""
import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I
from gpu_util import cuda_or_skip, dev
from fp32_bars import check as check32

pytestmark = pytest.mark.gpu

NO_SYMMETRIC = 8


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _run(torch, C, pts, kernel, w, n, N0, schedule, precision=None):
    prec = C.FP32_BULK if precision is None else precision
    P = C.plan_create(dev(torch, pts), kernel, n, 0.7, N0, precision=prec, max_nrhs=1,
                      no_persistent=True, schedule=schedule)
    out = C.evaluate(P, dev(torch, np.atleast_2d(w))).cpu().numpy()
    C.plan_sync(P)
    return C.plan_stats(P), out


# degree 8, 12 and 14: P = 81, 169, 225 proxies, i.e. each of the three row
# shapes of the pair kernel (2, 3 and 4 packed row pairs per lane)
CASES = [
    (O.KERNEL_LAPLACE, 8, 64),
    (O.KERNEL_NEWTON, 12, 144),
    (O.KERNEL_SAL, 8, 64),
    (O.KERNEL_BIHARMONIC, 14, 196),
    (O.KERNEL_ONE, 12, 144),
]


@pytest.mark.parametrize("kernel,n,N0", CASES)
def test_cc_pairs_match_the_oracle(kernel, n, N0):
    torch = cuda_or_skip()
    from paper_2508_13550_gb300 import csfmm as C
    pts, A = I.cubed_sphere_grid(48)
    coeffs = I.random_sh_coeffs(8, 1, seed=60 + kernel)
    f = I.sph_harm_combination(pts, coeffs, nrhs=1)[0]
    if kernel == O.KERNEL_ONE:
        # K = 1 sums the weights: zero-mean weights would leave a result 1e4
        # times smaller than sum |w|, i.e. only FP32 rounding, in either form
        f = f + 2.0 * np.abs(f).max()
    w = f * A
    ref = O.FMM(pts, n, 0.7, N0).evaluate(kernel, w[None, :])[0]
    st, out = _run(torch, C, pts, kernel, w, n, N0, 0)
    st_d, out_d = _run(torch, C, pts, kernel, w, n, N0, NO_SYMMETRIC)
    assert st["cc_sym_pairs"] > 0
    # every pair stands for two CC entries
    assert 2 * st["cc_sym_pairs"] <= st["n_list"][3]
    check32(f"fmm32-ccsym-k{kernel}-n{n}", _rel(out[0], ref))
    check32(f"fmm32-ccsym-vs-direct-k{kernel}-n{n}", _rel(out[0], out_d[0]))


def test_cc_pairs_on_an_unbalanced_tree():
    """Random points with a dense cap: the two traversal orders resolve some
    regions at different levels, so part of the CC entries have no mirror
    and stay with the direct evaluation beside the pairs."""
    torch = cuda_or_skip()
    from paper_2508_13550_gb300 import csfmm as C
    rng = np.random.default_rng(61)
    a = I.random_sphere_points(12000, 62)
    cap = a[a[:, 2] > 0.8]
    pts = np.concatenate([a, cap + 1e-3 * rng.standard_normal(cap.shape)])
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    w = rng.uniform(-1.0, 1.0, len(pts)) / len(pts)
    ref = O.FMM(pts, 8, 0.7, 64).evaluate(O.KERNEL_NEWTON, w[None, :])[0]
    st, out = _run(torch, C, pts, O.KERNEL_NEWTON, w, 8, 64, 0)
    _, out_d = _run(torch, C, pts, O.KERNEL_NEWTON, w, 8, 64, NO_SYMMETRIC)
    assert 0 < 2 * st["cc_sym_pairs"] < st["n_list"][3]
    print(f"\ndirect evaluation of every PP and CC entry: {_rel(out_d[0], ref):.3e}")
    check32("fmm32-ccsym-unbalanced-k2", _rel(out[0], ref))
    check32("fmm32-ccsym-vs-direct-unbalanced-k2", _rel(out[0], out_d[0]))


def test_no_cc_pairs_where_the_symmetric_pass_does_not_run():
    """FP64 plans and the Biot-Savart kernel (a vector kernel, odd in x - y)
    build no pairs."""
    torch = cuda_or_skip()
    from paper_2508_13550_gb300 import csfmm as C
    pts, A = I.cubed_sphere_grid(32)
    w = A.copy()
    st64, _ = _run(torch, C, pts, O.KERNEL_NEWTON, w, 8, 64, 0, precision=C.FP64)
    assert st64["cc_sym_pairs"] == 0
    st_bs, _ = _run(torch, C, pts, O.KERNEL_BIOT_SAVART, w, 8, 64, 0)
    assert st_bs["cc_sym_pairs"] == 0


def _mirrored_pairs(t, s):
    """Pairs (T, S), T < S, with both (T, S) and (S, T) in one list."""
    es = set(zip(t.tolist(), s.tolist()))
    return sum(1 for a, b in es if a < b and (b, a) in es)


@pytest.mark.parametrize("name,mk,n,N0", [
    ("cubed m=48, n=8", lambda: I.cubed_sphere_grid(48)[0], 8, 64),
    ("random 20,000 points, n=6", lambda: I.random_sphere_points(20000, 63), 6, 60),
])
def test_pair_counts_equal_the_oracle_lists(name, mk, n, N0):
    """The plan's mirrored PP and CC pairs are exactly the pairs of mirrored
    entries in the oracle's lists (integer work: bit-exact)."""
    torch = cuda_or_skip()
    from paper_2508_13550_gb300 import csfmm as C
    pts = mk()
    f = O.FMM(pts, n, 0.7, N0)
    L = f.lists()
    st, _ = _run(torch, C, pts, O.KERNEL_NEWTON, np.ones(len(pts)) / len(pts), n, N0, 0)
    assert st["sym_pairs"] == _mirrored_pairs(*L[O.PP]), name
    assert st["cc_sym_pairs"] == _mirrored_pairs(*L[O.CC]), name
