"""GPU parity of the remeshing (csfmm_remesh) and of the remeshed vortex-method
step (csfmm_bve_step_remeshed) through the C ABI against the oracle
(oracle/bve.py) on the same seeded inputs.

Bars: remeshing and FP64 remeshed steps agree with the oracle to 1e-12 of
max|zeta| (same cells and stencils, the same weighted fit solved by Cholesky
on the GPU and by an SVD least-squares solver in the oracle); FP32-bulk
remeshed steps to 1e-7.
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


def grid(torch, C, level, field="rh"):
    x, z, A, off, nb = I.workload_bve(level, field, with_adjacency=True)
    G = C.remesh_grid_create(dev(torch, x), dev(torch, off), dev(torch, nb))
    return G, x, z, A, off, nb


@pytest.mark.parametrize("level,steps", [(4, 1), (3, 10), (3, 4), (2, 3), (5, 2)])
def test_remesh_matches_oracle(torch, C, level, steps):
    G, x, z, A, off, nb = grid(torch, C, level)
    xs, zs = B.integrate(x, z, A, DT, steps, OMEGA)
    ref = B.remesh(x, off, nb, xs, zs)
    got = C.remesh(G, dev(torch, xs), dev(torch, zs)).cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(zs).max()
    moved = np.linalg.norm(xs - x, axis=1).max() / np.linalg.norm(x[nb[0]] - x[0])
    print(f"\nlevel {level}, {steps} steps (moved up to {moved:.1f} spacings): max err {err:.2e}")
    assert err < 1e-12


CASES = [("direct", 0, None), ("CSFMM n=6, plan per step", 6, False),
         ("CSFMM n=6, grid plan reused", 6, True)]


@pytest.mark.parametrize("name,degree,reuse", CASES)
def test_remeshed_step_fp64_matches_oracle(torch, C, name, degree, reuse):
    G, x, z, A, off, nb = grid(torch, C, 4)
    ref = B.remeshed_step(x, off, nb, z, A, DT, OMEGA, degree, 0.7, 144 if degree else None)
    P = C.plan_create(dev(torch, x), C.KERNEL_BIOT_SAVART, degree, 0.7, 144) if reuse else None
    got = C.bve_step_remeshed(G, dev(torch, z), dev(torch, A), DT, OMEGA, degree, 0.7, 144,
                              C.FP64, grid_plan=P).cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(z).max()
    print(f"\n{name}: max err {err:.2e}")
    assert err < 1e-12


def test_remeshed_trajectory_fp64_matches_oracle(torch, C):
    G, x, z, A, off, nb = grid(torch, C, 3, field="gaussian")
    zr = z.copy()
    dz, dA = dev(torch, z), dev(torch, A)
    for _ in range(10):
        zr = B.remeshed_step(x, off, nb, zr, A, DT, OMEGA)
        dz = C.bve_step_remeshed(G, dz, dA, DT, OMEGA, 0, precision=C.FP64)
    err = np.abs(dz.cpu().numpy() - zr).max() / np.abs(z).max()
    print(f"\n10 remeshed steps, Gaussian vortex, level 3: max err {err:.2e}")
    assert err < 1e-11


def test_remeshed_step_fp32_bulk(torch, C):
    G, x, z, A, off, nb = grid(torch, C, 4)
    ref = B.remeshed_step(x, off, nb, z, A, DT, OMEGA, 6, 0.7, 144)
    got = C.bve_step_remeshed(G, dev(torch, z), dev(torch, A), DT, OMEGA, 6, 0.7, 144,
                              C.FP32_BULK).cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(z).max()
    print(f"\nFP32 bulk remeshed step: max err {err:.2e}")
    assert err < 1e-7


def test_overlapping_output_refused(torch, C):
    G, x, z, A, off, nb = grid(torch, C, 3)
    xs, zs = B.integrate(x, z, A, DT, 2, OMEGA)
    dxs, dzs = dev(torch, xs), dev(torch, zs)
    with pytest.raises(C.CsfmmError) as e:
        C.remesh(G, dxs, dzs, out=dzs)
    assert e.value.status == 1
    # the remeshed step may update zeta and the tracer in place (it remeshes
    # into its own scratch)
    dz, dq, dA = dev(torch, z), dev(torch, x[:, 2].copy()), dev(torch, A)
    a, b = C.bve_step_remeshed(G, dz, dA, DT, OMEGA, 0, tracer=dq)
    C.bve_step_remeshed(G, dz, dA, DT, OMEGA, 0, tracer=dq, zeta_out=dz, tracer_out=dq)
    torch.cuda.synchronize()
    assert torch.equal(a, dz) and torch.equal(b, dq)


def test_remesh_errors(torch, C):
    x, z, A, off, nb = I.workload_bve(2, with_adjacency=True)
    bad = nb.copy()
    bad[5] = len(x)
    with pytest.raises(C.CsfmmError) as e:
        C.remesh_grid_create(dev(torch, x), dev(torch, off), dev(torch, bad))
    assert e.value.status == 1
    off_s = x.copy()
    off_s[3] *= 1.01
    with pytest.raises(C.CsfmmError) as e:
        C.remesh_grid_create(dev(torch, off_s), dev(torch, off), dev(torch, nb))
    assert e.value.status == 2
    G = C.remesh_grid_create(dev(torch, x), dev(torch, off), dev(torch, nb))
    # every particle at one point: each stencil's data are collinear, the fit is singular
    same = np.repeat(x[:1], len(x), axis=0)
    with pytest.raises(C.CsfmmError) as e:
        C.remesh(G, dev(torch, same), dev(torch, z))
    assert e.value.status == 8
    # a plan of another kernel is refused as the grid plan
    P = C.plan_create(dev(torch, x), C.KERNEL_LAPLACE, 3, 0.7, 8)
    with pytest.raises(C.CsfmmError) as e:
        C.bve_step_remeshed(G, dev(torch, z), dev(torch, A), DT, OMEGA, 3, 0.7, 8, C.FP64,
                            grid_plan=P)
    assert e.value.status == 1
    # the grid still works after the errors
    xs, zs = B.integrate(x, z, A, DT, 1, OMEGA)
    got = C.remesh(G, dev(torch, xs), dev(torch, zs)).cpu().numpy()
    assert np.abs(got - B.remesh(x, off, nb, xs, zs)).max() < 1e-12 * np.abs(zs).max()


def test_remesh_three_fields_matches_oracle(torch, C):
    G, x, z, A, off, nb = grid(torch, C, 3)
    xs, zs = B.integrate(x, z, A, DT, 6, OMEGA)
    F = np.stack([zs, xs[:, 2], np.cos(2 * xs[:, 0]) * xs[:, 1]])
    ref = B.remesh(x, off, nb, xs, F)
    got = C.remesh(G, dev(torch, xs), dev(torch, F)).cpu().numpy()
    assert np.abs(got - ref).max() < 1e-12 * np.abs(F).max()


def test_remeshed_tracer_trajectory_matches_oracle(torch, C):
    """Sec. 12 passive tracer q = z carried by the particles and remeshed with
    the vorticity: 8 remeshed steps, FP64 CSFMM velocity."""
    G, x, z, A, off, nb = grid(torch, C, 3)
    zr, qr = z.copy(), x[:, 2].copy()
    dz, dq, dA = dev(torch, z), dev(torch, x[:, 2].copy()), dev(torch, A)
    P = C.plan_create(dev(torch, x), C.KERNEL_BIOT_SAVART, 5, 0.7, 50)
    for _ in range(8):
        zr, qr = B.remeshed_step(x, off, nb, zr, A, DT, OMEGA, 5, 0.7, 50, tracer=qr)
        dz, dq = C.bve_step_remeshed(G, dz, dA, DT, OMEGA, 5, 0.7, 50, C.FP64, grid_plan=P,
                                     tracer=dq)
    ez = np.abs(dz.cpu().numpy() - zr).max() / np.abs(z).max()
    eq = np.abs(dq.cpu().numpy() - qr).max()
    print(f"\n8 remeshed steps with tracer: zeta err {ez:.2e}, tracer err {eq:.2e}")
    assert ez < 1e-11 and eq < 1e-11


@pytest.mark.parametrize("grid_kind", ["icosahedral", "variable"])
def test_remesh_random_moves_matches_oracle(torch, C, grid_kind):
    """Particles moved by seeded random tangent steps of up to 0.9 of the local
    spacing: many cross cell boundaries and data-disc edges in every direction.
    On the Schmidt-mapped grid (a conformal map, so the mapped triangulation
    stays Delaunay) spacings and cell radii vary 4x over the sphere, which
    exercises stencils sized and pruned per grid point."""
    level = 4
    verts, faces = I.icosahedral_triangulation(level)
    x = verts if grid_kind == "icosahedral" else I.schmidt_transform(verts, 0.5)
    off, nb = I.grid_adjacency(faces, len(x))
    h = np.array([np.linalg.norm(x[nb[off[k]:off[k + 1]]] - x[k], axis=1).min()
                  for k in range(len(x))])
    rng = np.random.default_rng(I.MASTER_SEED + 71)
    d = rng.normal(size=x.shape)
    d -= (d * x).sum(1, keepdims=True) * x
    d *= (0.9 * h * rng.uniform(size=len(x)) / np.linalg.norm(d, axis=1))[:, None]
    xs = x + d
    xs /= np.linalg.norm(xs, axis=1, keepdims=True)
    f = np.stack([I.rossby_haurwitz_vorticity(xs), np.cos(3 * xs[:, 0]) * xs[:, 2]])
    G = C.remesh_grid_create(dev(torch, x), dev(torch, off), dev(torch, nb))
    got = C.remesh(G, dev(torch, xs), dev(torch, f)).cpu().numpy()
    for q in range(2):
        ref = B.remesh(x, off, nb, xs, f[q])
        err = np.abs(got[q] - ref).max() / np.abs(f[q]).max()
        print(f"\n{grid_kind} level {level}, field {q}: max err {err:.2e}")
        assert err < 1e-12
