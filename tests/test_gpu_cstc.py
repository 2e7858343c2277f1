"""GPU parity of the cubed sphere tree code (Algorithm "CSTC") through the C
ABI against the oracle's CSTC on the same seeded inputs.

Bars: FP64 form vs oracle CSTC, relative l2 <= 1e-12 (same decisions, same
arithmetic in another rounding order); FP32 form vs oracle CSTC at most the
per-case bar of fp32_bars.py (about 4x the error measured on GB300); K = 1
reproduces sum_{j != i} w_j.
"""
import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I
from gpu_util import cuda_or_skip, dev
from fp32_bars import check as check32

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def C():
    from paper_2508_13550_gb300 import csfmm
    return csfmm


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def gpu_cstc(torch, C, pts, kernel, W, n, theta, N0, precision):
    P = C.plan_create(dev(torch, pts), kernel, n, theta, N0, precision=precision,
                      max_nrhs=max(1, np.atleast_2d(W).shape[0]))
    out = C.evaluate_cstc(P, dev(torch, np.atleast_2d(W)))
    torch.cuda.synchronize()
    C.plan_sync(P)
    res = out.cpu().numpy()
    C.plan_destroy(P)
    return res


def clustered(n, seed):
    rng = np.random.default_rng(seed)
    c = np.ones(3) / np.sqrt(3.0)
    v = rng.standard_normal((n, 3))
    v -= np.outer(v @ c, c)
    v /= np.linalg.norm(v, axis=1)[:, None]
    th = 0.3 * np.sqrt(rng.random(n))
    return np.vstack([np.cos(th)[:, None] * c + np.sin(th)[:, None] * v,
                      I.random_sphere_points(n // 4, seed + 1)])


CASES = [
    ("Poisson Y43, cubed m=32, n=8, N0=64", O.KERNEL_LAPLACE, lambda: I.workload_poisson_y43(32)[0], 8, 0.7, 64),
    ("Newtonian, random 20,000, n=6, N0=40", O.KERNEL_NEWTON, lambda: I.random_sphere_points(20000, 3), 6, 0.7, 40),
    ("Biot-Savart, cubed m=48, n=5, N0=30", O.KERNEL_BIOT_SAVART, lambda: I.cubed_sphere_grid(48)[0], 5, 0.7, 30),
    ("Laplace, clustered 6,000 + 1,500, n=4, N0=20, MAC 0.8", O.KERNEL_LAPLACE, lambda: clustered(6000, 4), 4, 0.8, 20),
    ("Newtonian, random 3,001, n=3, N0=1, MAC 0.9", O.KERNEL_NEWTON, lambda: I.random_sphere_points(3001, 5), 3, 0.9, 1),
    ("biharmonic, cubed m=32, n=6, N0=64", O.KERNEL_BIHARMONIC, lambda: I.cubed_sphere_grid(32)[0], 6, 0.7, 64),
]


@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
def test_cstc_matches_oracle(torch, C, case):
    name, kernel, mk, n, theta, N0 = CASES[case]
    pts = mk()
    rng = np.random.default_rng(8)
    W = rng.standard_normal((2, len(pts))) / len(pts)
    ref = O.FMM(pts, n, theta, N0).evaluate_cstc(kernel, W)
    g64 = gpu_cstc(torch, C, pts, kernel, W, n, theta, N0, C.FP64)
    assert rel(g64, ref) <= TOL64, (name, rel(g64, ref))
    g32 = gpu_cstc(torch, C, pts, kernel, W, n, theta, N0, C.FP32_BULK)
    check32(f"cstc32-case{case}", rel(g32, ref))


@pytest.mark.parametrize("precision", [0, 1])
def test_cstc_constant_kernel_covers_every_source_once(torch, C, precision):
    pts = I.random_sphere_points(12000, 6)
    w = np.random.default_rng(1).standard_normal(len(pts))
    g = gpu_cstc(torch, C, pts, O.KERNEL_ONE, w, 4, 0.7, 25, precision)[0, :, 0]
    err = np.max(np.abs(g - (w.sum() - w))) / np.abs(w).sum()
    if precision == 0:
        assert err <= 1e-12
    else:
        check32("cstc32-k1-max-over-sum-abs-w", err)


def test_cstc_config2_biot_savart_sampled(torch, C):
    """Biot-Savart on 6 x 256^2 = 393,216 cubed-sphere points (the RH-wave
    workload), n = 10, MAC 0.7, N0 = 400: FP64 CSTC against the oracle CSTC on
    400 sampled targets."""
    pts, A, w, _ = I.workload_rh_biot_savart(256)
    tg = np.sort(np.random.default_rng(3).choice(len(pts), 400, replace=False))
    ref = O.FMM(pts, 10, 0.7, 400).evaluate_cstc(O.KERNEL_BIOT_SAVART, w, targets=tg)
    g = gpu_cstc(torch, C, pts, O.KERNEL_BIOT_SAVART, w, 10, 0.7, 400, C.FP64)
    assert rel(g[:, tg], ref) <= TOL64


def test_cstc_and_fmm_agree_on_gpu(torch, C):
    """Both fast sums on one GPU plan approximate the same direct sum: the
    CSFMM within its truncation error at n = 8, the CSTC (looser
    particle-cluster separation test) within 1e-5."""
    pts, A, w, ex = I.workload_poisson_y43(64)
    P = C.plan_create(dev(torch, pts), O.KERNEL_LAPLACE, 8, 0.7, 64, precision=C.FP64)
    dw = dev(torch, w)
    fm = C.evaluate(P, dw)[0, :, 0].cpu().numpy()
    cs = C.evaluate_cstc(P, dw)[0, :, 0].cpu().numpy()
    C.plan_destroy(P)
    ds = O.direct(pts, O.KERNEL_LAPLACE, w)[0, :, 0]
    e_fm, e_cs = rel(fm, ds), rel(cs, ds)
    assert e_fm < 1e-7 and e_cs < 1e-5, (e_fm, e_cs)
