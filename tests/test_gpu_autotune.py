"""The autotuner picks a leaf size, then the launch schedule and tile shapes,
from timed evaluations, keeps the error within the stated factor of the
default's, and caches the choice."""
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
    assert r["from_cache"] == 0 and r["candidates"] >= 6
    if precision == 1 and nrhs >= 8:
        assert r["candidates"] >= 5 + 25  # leaf sizes, then schedules and tile shapes
    assert r["no_persistent"] in (0, 1) and 0 <= r["schedule"] <= 63
    assert r["max_leaf"] in {n * n * k for k in (1, 2, 3, 4, 6, 8)}
    assert r["rel_err"] <= 2.0 * r["default_rel_err"] + 1e-300
    assert r["ms_per_eval"] <= r["default_ms"]
    assert 0 < r["default_rel_err"] < 1e-4
    assert os.path.exists(cache)
    again = C.autotune(dev(torch, pts), C.KERNEL_LAPLACE, n, 0.7, dev(torch, W),
                       precision=precision, cache_path=cache)
    assert again["from_cache"] == 1 and again["max_leaf"] == r["max_leaf"]
    assert again["rhs_chunk"] == r["rhs_chunk"]
    assert (again["no_persistent"], again["schedule"]) == (r["no_persistent"], r["schedule"])
    # the chosen configuration builds and runs
    P = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, n, 0.7, r["max_leaf"],
                      precision=precision, max_nrhs=nrhs, rhs_chunk=r["rhs_chunk"],
                      no_persistent=r["no_persistent"], schedule=r["schedule"])
    out = C.evaluate(P, dev(torch, W)).cpu().numpy()
    assert np.isfinite(out).all()


@pytest.mark.parametrize("schedule", [1, 2, 4, 7, 8, 16, 24, 32, 40])
def test_every_schedule_matches_the_oracle(schedule):
    """Each tile shape and launch schedule the autotuner may pick computes the
    same sums: against the oracle FMM on the same tree within the FP32 bar of
    the default schedule (chunk width 16 changes only the rounding), and bit
    for bit equal to the default where only the work layout changes."""
    torch = cuda_or_skip()
    import oracle as O
    from paper_2508_13550_gb300 import csfmm as C
    from fp32_bars import check as check32
    pts, A = I.cubed_sphere_grid(48)
    nrhs = 16 if schedule < 8 else 1
    coeffs = I.random_sh_coeffs(6, nrhs, seed=1)
    W = I.sph_harm_combination(pts, coeffs, nrhs=nrhs) * A[None, :]
    ref = O.FMM(pts, 8, 0.7, 64).evaluate(O.KERNEL_LAPLACE, W)
    outs = []
    for sch in (0, schedule):
        P = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, 8, 0.7, 64, precision=C.FP32_BULK,
                          max_nrhs=nrhs, no_persistent=True, schedule=sch)
        outs.append(C.evaluate(P, dev(torch, W)).cpu().numpy())
        C.plan_sync(P)
    rel = max(float(np.linalg.norm(outs[1][r] - ref[r]) / np.linalg.norm(ref[r]))
              for r in range(nrhs))
    check32("fmm32-multi-k0-r16" if nrhs == 16 else "fmm32-schedule-k0-r1", rel)
    if not schedule & 4 and not schedule & 8:  # same arithmetic in another layout
        assert np.array_equal(outs[0], outs[1])
