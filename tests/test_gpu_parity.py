"""GPU parity tests: the CUDA library through the C ABI against the CPU oracle
on the same seeded inputs.

Bars (written here; each follows from the arithmetic on the two sides):
  - tree, tree order, cell centres and radii: identical (bitwise);
  - interaction lists: identical as sets per type;
  - FP64 FMM vs oracle FMM: relative l2 <= 1e-12;
  - FP64 direct sum vs oracle direct sum: relative l2 <= 1e-13;
  - FP32-bulk FMM and direct sum: relative l2 error against the oracle (its
    FP64 direct sum, or its FP64 FMM on the same tree, degree and MAC) at most
    the per-case bar of fp32_bars.py (about 4x the error measured on GB300).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I
from gpu_util import cuda_or_skip, dev, cell_keys
from fp32_bars import check as check32

pytestmark = pytest.mark.gpu

TOL_FMM64 = 1e-12
TOL_DS64 = 1e-13


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def C():
    from paper_2508_13550_gb300 import csfmm
    return csfmm


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def run_fmm(torch, C, pts, kernel, w, n, theta, N0, precision=0, max_nrhs=16):
    P = C.plan_create(dev(torch, pts), kernel, n, theta, N0, precision=precision,
                      max_nrhs=max_nrhs)
    out = C.evaluate(P, dev(torch, np.atleast_2d(w)))
    torch.cuda.synchronize()
    C.plan_sync(P)
    return P, out.cpu().numpy()


TREE_CASES = [
    ("cubed m=32 (6,144 points), n=8, N0=64", lambda: I.cubed_sphere_grid(32)[0], 8, 0.7, 64),
    ("random 5,000 points, n=4, N0=30", lambda: I.random_sphere_points(5000, 3), 4, 0.7, 30),
    ("shuffled cubed m=64, n=5, N0=40, MAC 0.5",
     lambda: I.cubed_sphere_grid(64, shuffle_seed=9)[0], 5, 0.5, 40),
    ("random 3,001 points, n=3, N0=1, MAC 0.9", lambda: I.random_sphere_points(3001, 4), 3, 0.9, 1),
    ("icosahedral 10,242 points, n=6, N0=144", lambda: I.icosahedral_grid(5)[0], 6, 0.7, 144),
    ("latitude-longitude 16,200 points, n=5, N0=40", lambda: I.latlon_grid(5)[0], 5, 0.7, 40),
]


@pytest.mark.parametrize("name,mk,n,theta,N0", TREE_CASES, ids=[c[0] for c in TREE_CASES])
def test_tree_and_lists_identical_to_oracle(torch, C, name, mk, n, theta, N0):
    pts = mk()
    ref = O.FMM(pts, n, theta, N0)
    P = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, n, theta, N0)
    st = C.plan_stats(P)
    info = ref.info()
    assert (st["ncells"], st["nleaves"], st["nlevels"]) == (info["ncells"], info["nleaves"],
                                                          info["nlevels"])
    assert np.array_equal(C.plan_export_order(P), ref.order())
    g, o = C.plan_export_cells(P), ref.cells()
    gk, ok = cell_keys(g), cell_keys(o)
    assert sorted(gk) == sorted(ok)
    gi = {k: i for i, k in enumerate(gk)}
    perm = np.array([gi[k] for k in ok])  # oracle cell -> gpu cell
    for f in ("begin", "end"):
        assert np.array_equal(g[f][perm], o[f]), f
    assert np.array_equal(g["centre"][perm], o["centre"])  # bitwise
    assert np.array_equal(g["radius"][perm], o["radius"])
    gpar = np.where(g["parent"][perm] >= 0, 0, -1)
    assert np.array_equal(gpar, np.where(o["parent"] >= 0, 0, -1))
    inv = np.empty(len(perm), dtype=np.int64)
    inv[perm] = np.arange(len(perm))  # gpu cell -> oracle cell
    for ty, (t_o, s_o) in ref.lists().items():
        t_g, s_g = C.plan_export_list(P, ty)
        assert sorted(zip(t_o.tolist(), s_o.tolist())) == sorted(
            zip(inv[t_g].tolist(), inv[s_g].tolist())), ty
    assert st["pairs_covered"] == len(pts) ** 2
    assert st["evals"][0] + st["evals"][1] + st["evals"][2] + st["evals"][3] == info["evals"]
    assert st["mac_margin"] == pytest.approx(info["margin"], rel=1e-12)


FMM_CASES = [
    # name, points, kernel, n, theta, N0, nrhs
    ("Laplace Y43 m=32 n=8 N0=64", "y43_32", O.KERNEL_LAPLACE, 8, 0.7, 64),
    ("Newton m=32 n=6 N0=20", "y43_32", O.KERNEL_NEWTON, 6, 0.7, 20),
    ("Biot-Savart RH m=48 n=7 N0=50", "rh_48", O.KERNEL_BIOT_SAVART, 7, 0.7, 50),
    ("Laplace random 7,777 n=5 N0=37 MAC 0.5", "rand_7777", O.KERNEL_LAPLACE, 5, 0.5, 37),
    ("Newton random 7,777 n=9 N0=100 MAC 0.9", "rand_7777", O.KERNEL_NEWTON, 9, 0.9, 100),
    ("K=1 random 7,777 n=3 N0=12", "rand_7777", O.KERNEL_ONE, 3, 0.7, 12),
    ("Laplace degree 1 m=16 N0=8", "y43_16", O.KERNEL_LAPLACE, 1, 0.7, 8),
    ("Laplace degree 16 m=32 N0=64", "y43_32", O.KERNEL_LAPLACE, 16, 0.7, 64),
    ("Laplace Y43 icosahedral 40,962 n=6 N0=144", "ico_6", O.KERNEL_LAPLACE, 6, 0.7, 144),
    ("biharmonic Y43 m=32 n=8 N0=64", "y43_32", O.KERNEL_BIHARMONIC, 8, 0.7, 64),
    ("biharmonic random 7,777 n=5 N0=37 MAC 0.5", "rand_7777", O.KERNEL_BIHARMONIC, 5, 0.5, 37),
    ("Biot-Savart RH latitude-longitude 16,200 n=6 N0=60", "latlon_5", O.KERNEL_BIOT_SAVART, 6, 0.7, 60),
]


def _points(tag):
    if tag.startswith("y43_"):
        m = int(tag[4:])
        pts, A = I.cubed_sphere_grid(m)
        return pts, I.real_sph_harm(4, 3, pts) * A
    if tag.startswith("rh_"):
        m = int(tag[3:])
        pts, A = I.cubed_sphere_grid(m)
        return pts, I.rossby_haurwitz_vorticity(pts) * A
    if tag.startswith("ico_"):
        pts, A = I.icosahedral_grid(int(tag[4:]))
        return pts, I.real_sph_harm(4, 3, pts) * A
    if tag.startswith("latlon_"):
        pts, A = I.latlon_grid(int(tag[7:]))
        return pts, I.rossby_haurwitz_vorticity(pts) * A
    N = int(tag.split("_")[1])
    pts = I.random_sphere_points(N, 17)
    return pts, np.random.default_rng(18).standard_normal(N) * (4 * math.pi / N)


@pytest.mark.parametrize("name,tag,kernel,n,theta,N0", FMM_CASES, ids=[c[0] for c in FMM_CASES])
def test_fp64_fmm_matches_oracle_fmm(torch, C, name, tag, kernel, n, theta, N0):
    pts, w = _points(tag)
    rng = np.random.default_rng(5)
    W = np.stack([w, rng.standard_normal(len(w)) * np.abs(w).mean(), 2 * w, -w, 0.5 * w])
    ref = O.FMM(pts, n, theta, N0).evaluate(kernel, W)
    _, got = run_fmm(torch, C, pts, kernel, W, n, theta, N0)
    for r in range(W.shape[0]):
        assert rel(got[r], ref[r]) <= TOL_FMM64, (r, rel(got[r], ref[r]))
    if kernel == O.KERNEL_ONE:
        exact = W.sum(axis=1, keepdims=True) - W
        assert np.max(np.abs(got[:, :, 0] - exact)) < 1e-12


def test_fp64_fmm_config2_biot_savart_full(torch, C):
    """Rossby-Haurwitz Biot-Savart workload, 6 x 256^2 = 393,216 points, n=10,
    MAC 0.7, N0=400 (the paper's default 4 n^2): every output."""
    pts, A, w, _ = I.workload_rh_biot_savart(256)
    ref = O.FMM(pts, 10, 0.7, 400).evaluate(O.KERNEL_BIOT_SAVART, w)
    _, got = run_fmm(torch, C, pts, O.KERNEL_BIOT_SAVART, w, 10, 0.7, 400)
    assert rel(got[0], ref[0]) <= TOL_FMM64


def test_fmm_multi_rhs_consistent_with_single(torch, C):
    pts, w = _points("rand_7777")
    rng = np.random.default_rng(2)
    W = rng.standard_normal((7, len(w)))
    P = C.plan_create(dev(torch, pts), C.KERNEL_NEWTON, 5, 0.7, 40, max_nrhs=3)
    allr = C.evaluate(P, dev(torch, W)).cpu().numpy()
    for r in range(7):
        one = C.evaluate(P, dev(torch, W[r:r + 1])).cpu().numpy()
        assert np.array_equal(one[0], allr[r])
    host = C.evaluate_host(P, W)
    assert np.array_equal(host, allr)
    ws = C.workspace_create(P, 4)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        other = C.evaluate_ws(P, ws, dev(torch, W), stream=s.cuda_stream)
    s.synchronize()
    assert np.array_equal(other.cpu().numpy(), allr)
    C.workspace_destroy(ws)


@pytest.mark.parametrize("kernel", [O.KERNEL_LAPLACE, O.KERNEL_BIOT_SAVART, O.KERNEL_NEWTON,
                                    O.KERNEL_BIHARMONIC, O.KERNEL_ONE])
def test_direct_matches_oracle(torch, C, kernel):
    pts = I.random_sphere_points(3001, 8)
    W = np.random.default_rng(9).standard_normal((5, 3001))
    ref = O.direct(pts, kernel, W)
    got = C.direct(dev(torch, pts), kernel, dev(torch, W)).cpu().numpy()
    for r in range(5):
        assert rel(got[r], ref[r]) <= TOL_DS64
    tg = np.array([0, 5, 3000, 17, 5], dtype=np.int64)
    sub = C.direct(dev(torch, pts), kernel, dev(torch, W), targets=dev(torch, tg)).cpu().numpy()
    assert rel(sub, ref[:, tg]) <= TOL_DS64
    g32 = C.direct(dev(torch, pts), kernel, dev(torch, W), precision=C.FP32_BULK).cpu().numpy()
    check32(f"direct32-k{kernel}", rel(g32, ref))


def test_fp32_bulk_error_against_fp64_direct(torch, C):
    """FP32-bulk FMM error E(FS32, DS64) next to the FP64 truncation error
    E(FS64, DS64), Poisson Y43 on 6 x 64^2 points, n=8, MAC 0.7."""
    pts, A, w, ex = I.workload_poisson_y43(64)
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    _, f64 = run_fmm(torch, C, pts, O.KERNEL_LAPLACE, w, 8, 0.7, 64)
    _, f32 = run_fmm(torch, C, pts, O.KERNEL_LAPLACE, w, 8, 0.7, 64, precision=C.FP32_BULK)
    e64 = O.rel_l2(f64[0, :, 0], ds, A, ex[0])
    e32 = O.rel_l2(f32[0, :, 0], ds, A, ex[0])
    print(f"\nE(FS64,DS)={e64:.3e}  E(FS32,DS)={e32:.3e}")
    assert e64 < 1e-7
    check32("fmm32-poisson-y43-m64-n8", e32)


def test_full_size_newton_config_sampled(torch, C):
    """The benchmark's workload: Newtonian kernel, land-masked field on
    6 x 1024^2 = 6,291,456 points, n=12, MAC 0.7, N0=576.  The FP64 path is
    compared with the oracle FMM on 600 sampled targets; the FP32-bulk path
    (the benchmarked form) with the oracle direct sum on 300 targets."""
    pts, A, w = I.workload_newton_land(1024)
    N = len(pts)
    tg = np.sort(np.random.default_rng(11).choice(N, 600, replace=False))
    ref = O.FMM(pts, 12, 0.7, 576)
    ref_s = ref.evaluate(O.KERNEL_NEWTON, w, tg)[0, :, 0]
    P64, f64 = run_fmm(torch, C, pts, O.KERNEL_NEWTON, w, 12, 0.7, 576)
    assert rel(f64[0, tg, 0], ref_s) <= TOL_FMM64
    st = C.plan_stats(P64)
    assert sum(st["evals"]) == ref.info()["evals"]
    del P64
    _, f32 = run_fmm(torch, C, pts, O.KERNEL_NEWTON, w, 12, 0.7, 576, precision=C.FP32_BULK)
    tg2 = tg[:300]
    ds = O.direct(pts, O.KERNEL_NEWTON, w, tg2)[0, :, 0]
    e32 = rel(f32[0, tg2, 0], ds)
    e64 = rel(f64[0, tg2, 0], ds)
    print(f"\nconfig-3 sample: E(FS64,DS)={e64:.3e}  E(FS32,DS)={e32:.3e}")
    assert e64 < 1e-8
    check32("fmm32-newton-land-6m-n12", e32)


def test_full_size_multi_rhs_config_sampled(torch, C):
    """The multi-RHS workload at full size: Poisson kernel, 6 x 512^2 =
    1,572,864 points, 16 right-hand sides, n=10, MAC 0.7, N0=400, FP32 bulk in
    the launch configuration the benchmark times (16 RHS per kernel value).
    Every right-hand side is compared with the oracle direct sum on 64
    sampled targets, and with the FP64 CSFMM of the same plan shape."""
    pts, A, W, _ = I.workload_multi_rhs(512, 16, with_exact=False)
    N = len(pts)
    tg = np.sort(np.random.default_rng(12).choice(N, 64, replace=False))
    ds = O.direct(pts, O.KERNEL_LAPLACE, W, tg)[:, :, 0]
    P = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, 10, 0.7, 400, precision=C.FP32_BULK,
                      max_nrhs=16)
    f32 = C.evaluate(P, dev(torch, W)).cpu().numpy()[:, tg, 0]
    del P
    errs = [rel(f32[r], ds[r]) for r in range(16)]
    print(f"\nconfig-4 sample: max over 16 RHS of E(FS32,DS) = {max(errs):.3e}")
    check32("fmm32-poisson16-1.5m-n10", max(errs))
    P64 = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, 10, 0.7, 400, max_nrhs=4)
    f64 = C.evaluate(P64, dev(torch, W[:4])).cpu().numpy()[:, tg, 0]
    for r in range(4):
        assert rel(f64[r], ds[r]) < 1e-8


def test_edge_cases(torch, C):
    # one point: no sources, phi = 0
    p1 = np.array([[0.0, 0.0, 1.0]])
    _, out = run_fmm(torch, C, p1, C.KERNEL_LAPLACE, np.array([2.0]), 4, 0.7, 10)
    assert out.shape == (1, 1, 1) and out[0, 0, 0] == 0.0
    # two points on different faces
    p2 = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    _, out = run_fmm(torch, C, p2, C.KERNEL_NEWTON, np.array([1.0, 3.0]), 2, 0.7, 1)
    assert np.allclose(out[0, :, 0], [3 / math.sqrt(2), 1 / math.sqrt(2)], rtol=1e-14)
    # clustered points (deep, non-uniform tree) against the oracle
    rng = np.random.default_rng(4)
    v = np.array([0.3, -0.2, 1.0]) + 0.01 * rng.standard_normal((2000, 3))
    pts = v / np.linalg.norm(v, axis=1, keepdims=True)
    w = rng.standard_normal(2000)
    ref = O.FMM(pts, 4, 0.7, 8).evaluate(C.KERNEL_LAPLACE, w)
    P, got = run_fmm(torch, C, pts, C.KERNEL_LAPLACE, w, 4, 0.7, 8)
    assert C.plan_stats(P)["nlevels"] > 8
    assert rel(got, ref) <= TOL_FMM64
    # N smaller than the leaf size: every face is one leaf
    pts = I.random_sphere_points(50, 3)
    w = rng.standard_normal(50)
    _, got = run_fmm(torch, C, pts, C.KERNEL_BIOT_SAVART, w, 3, 0.7, 100)
    ds = O.direct(pts, C.KERNEL_BIOT_SAVART, w)
    assert rel(got, ds) <= TOL_DS64


def test_argument_errors(torch, C):
    pts = dev(torch, I.random_sphere_points(100, 1))
    bad = [
        dict(kernel_id=7, degree=4, theta=0.7, max_leaf=10),
        dict(kernel_id=0, degree=0, theta=0.7, max_leaf=10),
        dict(kernel_id=0, degree=17, theta=0.7, max_leaf=10),
        dict(kernel_id=0, degree=4, theta=1.0, max_leaf=10),
        dict(kernel_id=0, degree=4, theta=0.0, max_leaf=10),
        dict(kernel_id=0, degree=4, theta=0.7, max_leaf=0),
    ]
    for kw in bad:
        with pytest.raises(C.CsfmmError) as e:
            C.plan_create(pts, kw["kernel_id"], kw["degree"], kw["theta"], kw["max_leaf"])
        assert e.value.status == 1
    off = I.random_sphere_points(100, 1)
    off[17] *= 1.001
    with pytest.raises(C.CsfmmError) as e:
        C.plan_create(dev(torch, off), 0, 4, 0.7, 10)
    assert e.value.status == 2
    nan = I.random_sphere_points(100, 1)
    nan[3, 1] = np.nan
    with pytest.raises(C.CsfmmError) as e:
        C.plan_create(dev(torch, nan), 0, 4, 0.7, 10)
    assert e.value.status == 2
    P = C.plan_create(pts, 0, 4, 0.7, 10)
    # host memory where device memory is required: the library itself refuses it
    import ctypes
    host_w = np.zeros((1, 100))
    out = torch.zeros((1, 100, 1), dtype=torch.float64, device="cuda")
    rc = C.load().csfmm_evaluate(P.handle, ctypes.c_void_p(host_w.ctypes.data), 1,
                                 ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1 and "device memory" in C.last_error()
    with pytest.raises(C.CsfmmError):
        C.direct(pts, 5, torch.zeros((1, 100), dtype=torch.float64, device="cuda"))
    # the library still works after the errors
    out = C.evaluate(P, torch.ones((1, 100), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert np.isfinite(out.cpu().numpy()).all()


@pytest.mark.parametrize("kernel,nrhs", [(O.KERNEL_LAPLACE, 16), (O.KERNEL_NEWTON, 9),
                                         (O.KERNEL_ONE, 8), (O.KERNEL_BIOT_SAVART, 6),
                                         (O.KERNEL_BIHARMONIC, 16)])
def test_fp32_multi_rhs_matches_oracle_and_single(torch, C, kernel, nrhs):
    """FP32-bulk with many right-hand sides (chunks of 16 / 8 share each kernel
    value) against the oracle FMM on the same tree, degree and MAC (so the
    difference is the FP32 rounding alone), element by element, and against
    one-at-a-time FP32 evaluations."""
    pts, A = I.cubed_sphere_grid(48)
    coeffs = I.random_sh_coeffs(6, nrhs, seed=kernel + 1)
    W = I.sph_harm_combination(pts, coeffs, nrhs=nrhs) * A[None, :]
    if kernel == O.KERNEL_ONE:
        # K = 1 sums all weights: keep that sum away from zero (no cancellation)
        W = W + A[None, :]
    ref = O.FMM(pts, 8, 0.7, 64).evaluate(kernel, W)
    P32 = C.plan_create(dev(torch, pts), kernel, 8, 0.7, 64, precision=C.FP32_BULK, max_nrhs=nrhs)
    dW = dev(torch, W)
    allr = C.evaluate(P32, dW).cpu().numpy()
    check32(f"fmm32-multi-k{kernel}-r{nrhs}", max(rel(allr[r], ref[r]) for r in range(nrhs)))
    worst = 0.0
    for r in range(nrhs):
        one = C.evaluate(P32, dW[r:r + 1].contiguous()).cpu().numpy()[0]
        worst = max(worst, rel(allr[r], one))
    check32(f"fmm32-chunk-vs-single-k{kernel}", worst)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_matches_direct_launches(torch, C, precision):
    """use_graphs: captured once per right-hand-side count, replayed with the
    caller's buffers retargeted; results equal plain launches bit for bit."""
    pts, A = I.cubed_sphere_grid(40)
    rng = np.random.default_rng(precision)
    plain = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, 7, 0.7, 50, precision=precision)
    graph = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, 7, 0.7, 50, precision=precision,
                          use_graphs=1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for call, nrhs in enumerate([1, 3, 1, 3, 2]):
            W = dev(torch, rng.standard_normal((nrhs, len(pts))) * A)
            ref = C.evaluate(plain, W, stream=s.cuda_stream)
            got = C.evaluate(graph, W, stream=s.cuda_stream)  # new buffers every call
            s.synchronize()
            assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy()), call
    C.plan_sync(graph, stream=s.cuda_stream)


@pytest.mark.parametrize("sign", ["positive", "mixed"])
@pytest.mark.parametrize("kernel", [O.KERNEL_NEWTON, O.KERNEL_LAPLACE, O.KERNEL_BIHARMONIC,
                                    O.KERNEL_ONE])
def test_fp32_symmetric_near_field(torch, C, kernel, sign):
    """One right-hand side in FP32 bulk evaluates mirrored PP leaf pairs once
    for both directions.  Compared element by element with the oracle FMM on
    the same tree, degree and MAC (the difference is the FP32 rounding alone),
    for a positive density and for zero-mean weights of mixed sign (whose sums
    cancel), and with the two-RHS launch, which evaluates every PP entry
    directly."""
    pts = I.random_sphere_points(20000, 31)
    rng = np.random.default_rng(32)
    if sign == "positive":
        w = rng.uniform(0.5, 1.5, len(pts)) * (4 * math.pi / len(pts))
    else:
        w = rng.standard_normal(len(pts)) * (4 * math.pi / len(pts))
        if kernel == O.KERNEL_ONE:
            w = w + 4 * math.pi / len(pts)  # K = 1 needs a sum away from zero
    P32 = C.plan_create(dev(torch, pts), kernel, 5, 0.7, 40, precision=C.FP32_BULK)
    st = C.plan_stats(P32)
    assert st["sym_pairs"] > 0.3 * st["n_list"][0] / 2
    one = C.evaluate(P32, dev(torch, w[None])).cpu().numpy()[0]
    two = C.evaluate(P32, dev(torch, np.stack([w, w]))).cpu().numpy()
    ref = O.FMM(pts, 5, 0.7, 40).evaluate(kernel, w)[0]
    check32(f"fmm32-sym-k{kernel}-{sign}", rel(one, ref))
    check32(f"fmm32-sym-vs-2rhs-k{kernel}-{sign}", rel(one, two[0]))


@pytest.mark.parametrize("kernel", [O.KERNEL_NEWTON, O.KERNEL_LAPLACE])
def test_full_size_symmetric_near_field_mixed_sign(torch, C, kernel):
    """The benchmarked launch shape (6 x 1024^2 = 6,291,456 cubed-sphere
    points, n = 12, MAC 0.7, N0 = 576, one right-hand side, FP32 bulk, so the
    mirrored-pair kernel carries most of the near field) on zero-mean weights
    of mixed sign: a seeded random combination of real harmonics Y_nm,
    n <= 16, plus white noise at 10% of its rms, times the cell areas.  The
    FP32-bulk potential is compared with the oracle direct sum on 256 sampled
    targets."""
    pts, A = I.cubed_sphere_grid(1024)
    N = len(pts)
    coeffs = I.random_sh_coeffs(16, 1, seed=40 + kernel)
    f = I.sph_harm_combination(pts, coeffs, nrhs=1)[0]
    f = f + 0.1 * np.sqrt(np.mean(f * f)) * np.random.default_rng(41).standard_normal(N)
    w = f * A
    tg = np.sort(np.random.default_rng(42 + kernel).choice(N, 256, replace=False))
    ds = O.direct(pts, kernel, w, tg)[0, :, 0]
    P32, f32 = run_fmm(torch, C, pts, kernel, w, 12, 0.7, 576, precision=C.FP32_BULK)
    st = C.plan_stats(P32)
    assert st["sym_evals"] > 0.5 * st["evals"][0] / 2
    del P32
    e32 = rel(f32[0, tg, 0], ds)
    check32(f"fmm32-sym-6m-mixed-k{kernel}", e32)
