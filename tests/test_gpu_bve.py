"""GPU parity of the vortex-method step for the barotropic vorticity equation
(csfmm_bve_step; Sec. 2.3, Eq. BVE_ODEs, RK4 as in Sec. 12) through the C ABI
against the oracle's RK4 integrator on the same seeded inputs.

Bars.  FP64 direct and FP64 CSFMM velocity: the step agrees with the oracle's
step to 1e-13 in the positions and 1e-12 max|zeta| in the vorticity (same
formulas, other rounding order; the CSFMM trees at the stage positions are the
same because the stage positions agree to rounding).  FP32-bulk CSFMM: within
dt times the FP32-bulk velocity error (about 1e-6 of |u|).
"""
import numpy as np
import pytest

import oracle.bve as B
from paper_2508_13550_gb300 import inputs as I
from gpu_util import cuda_or_skip, dev

pytestmark = pytest.mark.gpu

OMEGA = I.BVE_OMEGA
DT = I.BVE_DT


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def C():
    from paper_2508_13550_gb300 import csfmm
    return csfmm


def gpu_step(torch, C, x, z, A, degree, theta=0.7, N0=0, precision=0, steps=1):
    dx, dz, dA = dev(torch, x), dev(torch, z), dev(torch, A)
    for _ in range(steps):
        dx, dz = C.bve_step(dx, dz, dA, DT, OMEGA, degree, theta, N0, precision)
    torch.cuda.synchronize()
    return dx.cpu().numpy(), dz.cpu().numpy()


CASES = [
    ("icosahedral level 4, RH wave, direct", lambda: I.workload_bve(4), 0, 0.7, 0),
    ("icosahedral level 4, RH wave, n=6 MAC 0.7", lambda: I.workload_bve(4), 6, 0.7, 144),
    ("icosahedral level 3, Gaussian vortex, n=4 N0=8", lambda: I.workload_bve(3, "gaussian"),
     4, 0.8, 8),
    ("random 1500, Gaussian vortex, n=5 N0=20",
     lambda: (lambda p: (p, I.gaussian_vortex_vorticity(p), np.full(len(p), 4 * np.pi / len(p))))(
         I.random_sphere_points(1500, 11)), 5, 0.7, 20),
    ("icosahedral level 0 (12 particles), direct", lambda: I.workload_bve(0), 0, 0.7, 0),
    ("icosahedral level 0 (12 particles), n=2 N0=1", lambda: I.workload_bve(0), 2, 0.5, 1),
]


@pytest.mark.parametrize("name,mk,degree,theta,N0", CASES)
def test_step_fp64_matches_oracle(torch, C, name, mk, degree, theta, N0):
    x, z, A = mk()
    xo, zo = B.rk4_step(x, z, A, DT, OMEGA, degree, theta, N0 if N0 else None)
    xg, zg = gpu_step(torch, C, x, z, A, degree, theta, N0, C.FP64)
    ex = np.abs(xg - xo).max()
    ez = np.abs(zg - zo).max() / np.abs(z).max()
    print(f"\n{name}: |dx| {ex:.2e}  |dzeta|/max|zeta| {ez:.2e}  moved {np.abs(xo - x).max():.2e}")
    assert ex < 1e-13
    assert ez < 1e-12
    assert np.allclose(np.linalg.norm(xg, axis=1), 1.0, atol=4e-16)


def test_step_fp32_bulk_within_velocity_error(torch, C):
    x, z, A = I.workload_bve(4)
    xo, zo = B.rk4_step(x, z, A, DT, OMEGA, 6, 0.7, 144)
    xg, zg = gpu_step(torch, C, x, z, A, 6, 0.7, 144, C.FP32_BULK)
    moved = np.abs(xo - x).max()
    ex = np.abs(xg - xo).max()
    ez = np.abs(zg - zo).max() / np.abs(z).max()
    print(f"\nFP32 bulk: |dx| {ex:.2e} (moved {moved:.2e})  |dzeta|/max|zeta| {ez:.2e}")
    assert ex < 1e-6 * moved
    assert ez < 1e-7


def test_in_place_step_is_identical(torch, C):
    x, z, A = I.workload_bve(3)
    dx, dz, dA = dev(torch, x), dev(torch, z), dev(torch, A)
    xo, zo = C.bve_step(dx, dz, dA, DT, OMEGA, 5, 0.7, 50)
    C.bve_step(dx, dz, dA, DT, OMEGA, 5, 0.7, 50, x_out=dx, zeta_out=dz)
    torch.cuda.synchronize()
    assert torch.equal(dx, xo) and torch.equal(dz, zo)


def test_rh_wave_fmm_error_negligible_against_discretisation(torch, C):
    """Sec. 12: E_zeta with the CSFMM velocity is essentially that of the
    direct sum, and it falls about 4x from icosahedral level 4 (oracle,
    direct sum) to level 5 (GPU)."""
    steps = 10
    x4, z4, A4 = I.workload_bve(4)
    xo, zo = B.integrate(x4, z4, A4, DT, steps, OMEGA)
    e4 = B.vorticity_error(zo, I.rossby_haurwitz_vorticity(xo), A4)
    x, z, A = I.workload_bve(5)
    e = {}
    for tag, deg, prec in (("ds64", 0, C.FP64), ("fmm64", 6, C.FP64), ("fmm32", 6, C.FP32_BULK)):
        xg, zg = gpu_step(torch, C, x, z, A, deg, 0.7, 144, prec, steps=steps)
        e[tag] = B.vorticity_error(zg, I.rossby_haurwitz_vorticity(xg), A)
    print(f"\nE_zeta(0.1 day): level 4 oracle {e4:.3e}; level 5 GPU {e}")
    assert 3.0 < e4 / e["ds64"] < 5.0
    assert abs(e["fmm64"] - e["ds64"]) < 1e-3 * e["ds64"]
    assert abs(e["fmm32"] - e["ds64"]) < 1e-3 * e["ds64"]


def test_argument_errors(torch, C):
    x, z, A = I.workload_bve(1)
    dx, dz, dA = dev(torch, x), dev(torch, z), dev(torch, A)
    with pytest.raises(C.CsfmmError) as e:
        C.bve_step(dx, dz, dA, 0.0, OMEGA, 6)
    assert e.value.status == 1
    with pytest.raises(C.CsfmmError) as e:
        C.bve_step(dx, dz, dA, DT, OMEGA, -1)
    assert e.value.status == 1
    off = x.copy()
    off[5] *= 1.001
    with pytest.raises(C.CsfmmError) as e:
        C.bve_step(dev(torch, off), dz, dA, DT, OMEGA, 3, 0.7, 8)
    assert e.value.status == 2
