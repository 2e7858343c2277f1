"""The paper's own numbers on its own grid: Poisson problem on the
icosahedral grid with N = 655362 points (Table "grids", level 8), through the
C ABI (FP64 CSFMM and FP64 direct sum on sampled targets).

- Sec. 11 states that the CSFMM solution error for Y43 at N = 655362 is about
  4.4e-4 (it is the midpoint-rule discretization error, Fig. l2y43error);
- Table "csfmmerrors" lists E(phi_FS, phi_DS) per MAC and degree: at MAC 0.9
  and n = 2, 4 our tree, proxies and passes reproduce the entries for Y43 and
  Y85 to within 1.3x (bar 1.5x for the sampling of 8192 targets); elsewhere
  ours are at most that far above the paper's (smaller in most entries: the
  cluster radius here bounds the whole cell).
"""
import math

import numpy as np
import pytest

from paper_2508_13550_gb300 import inputs as I
from conftest import golden
from gpu_util import cuda_or_skip, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = cuda_or_skip()
    from paper_2508_13550_gb300 import csfmm as C
    pts, A = I.icosahedral_grid(8)
    assert len(pts) == 655362
    Y = np.stack([I.real_sph_harm(4, 3, pts), I.real_sph_harm(8, 5, pts)])
    EX = np.stack([Y[0] / 20.0, Y[1] / 72.0])
    W = np.ascontiguousarray(Y * A)
    tg = np.sort(np.random.default_rng(20250813).choice(len(pts), 8192, replace=False))
    dp, dW = dev(torch, pts), dev(torch, W)
    ds = C.direct(dp, C.KERNEL_LAPLACE, dW, precision=C.FP64,
                  targets=dev(torch, tg))[:, :, 0].cpu().numpy()
    At = A[tg]
    den = np.sum(EX[:, tg] ** 2 * At, axis=1)
    paper = {(r[0], float(r[1])): [float(x) for x in r[2:]]
             for r in golden("csfmm_errors_table.txt")}
    return torch, C, dp, dW, tg, ds, EX, At, den, paper


def test_discretization_error_matches_the_paper(setup):
    torch, C, dp, dW, tg, ds, EX, At, den, paper = setup
    e = np.sqrt(np.sum((ds - EX[:, tg]) ** 2 * At, axis=1) / den)
    assert abs(e[0] - 4.4e-4) < 0.05 * 4.4e-4, e[0]
    assert 1e-4 < e[0] < 1e-3 and 1e-4 < e[1] < 3e-3


@pytest.mark.parametrize("mac,n", [(0.9, 2), (0.9, 4), (0.9, 6), (0.7, 4), (0.7, 6), (0.5, 4)])
def test_fmm_error_against_table_csfmmerrors(setup, mac, n):
    torch, C, dp, dW, tg, ds, EX, At, den, paper = setup
    P = C.plan_create(dp, C.KERNEL_LAPLACE, n, mac, 4 * n * n, precision=C.FP64, max_nrhs=2)
    fs = C.evaluate(P, dW)[:, :, 0].cpu().numpy()[:, tg]
    C.plan_destroy(P)
    e = np.sqrt(np.sum((fs - ds) ** 2 * At, axis=1) / den)
    for k, name in enumerate(("Y43", "Y85")):
        ref = paper[(name, mac)][n // 2 - 1]
        assert e[k] <= 1.5 * ref, (name, mac, n, e[k], ref)
        if mac == 0.9 and n <= 4:
            assert e[k] >= ref / 1.5, (name, mac, n, e[k], ref)
