"""The autotuner picks a leaf size (and RHS chunk) from timed evaluations,
keeps the error within the stated factor of the default's, and caches it."""
import os

import numpy as np
import pytest

from paper_2508_13550_gb300 import inputs as I
from gpu_util import cuda_or_skip, dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,nrhs", [(0, 1), (1, 8)])
def test_autotune_choice_and_cache(tmp_path, precision, nrhs):
    torch = cuda_or_skip()
    from paper_2508_13550_gb300 import csfmm as C
    pts, A = I.cubed_sphere_grid(64)
    coeffs = I.random_sh_coeffs(6, nrhs, seed=4)
    W = I.sph_harm_combination(pts, coeffs, nrhs=nrhs) * A[None, :]
    cache = str(tmp_path / "tune.txt")
    n = 6
    r = C.autotune(dev(torch, pts), C.KERNEL_LAPLACE, n, 0.7, dev(torch, W), precision=precision,
                   cache_path=cache, err_factor=2.0)
    assert r["from_cache"] == 0 and r["candidates"] >= 5
    assert r["max_leaf"] in {n * n * k for k in (1, 2, 3, 4, 6, 8)}
    assert r["rel_err"] <= 2.0 * r["default_rel_err"] + 1e-300
    assert r["ms_per_eval"] <= r["default_ms"]
    assert 0 < r["default_rel_err"] < 1e-4
    assert os.path.exists(cache)
    again = C.autotune(dev(torch, pts), C.KERNEL_LAPLACE, n, 0.7, dev(torch, W),
                       precision=precision, cache_path=cache)
    assert again["from_cache"] == 1 and again["max_leaf"] == r["max_leaf"]
    assert again["rhs_chunk"] == r["rhs_chunk"]
    # the chosen configuration builds and runs
    P = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, n, 0.7, r["max_leaf"],
                      precision=precision, max_nrhs=nrhs, rhs_chunk=r["rhs_chunk"])
    out = C.evaluate(P, dev(torch, W)).cpu().numpy()
    assert np.isfinite(out).all()
