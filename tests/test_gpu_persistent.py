"""GPU tests of the persistent multi-right-hand-side launch (FP32 bulk,
scalar kernels, nrhs a multiple of 8): one kernel evaluates the far field,
the near field, L2L and L2P of every chunk of right-hand sides, drawing items
from a device work counter and waiting, bounded in time, for the downward
pass's dependencies.

Bars: the persistent launch runs the per-phase kernels' item functions with
the same per-target operation order, so its output equals the per-phase
launches bit for bit (also when replayed from a CUDA graph with new buffers);
its accuracy against the oracle is that of the per-phase launches (the FP32
multi-RHS parity tests of test_gpu_parity.py take this launch by default); a
wait that can never be satisfied (test hook) ends in CSFMM_ERR_TIMEOUT
after its bound, and the plan evaluates correctly afterwards.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_13550_gb300 import inputs as I
from gpu_util import cuda_or_skip, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def C():
    from paper_2508_13550_gb300 import csfmm
    return csfmm


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def _weights(pts, A, nrhs, seed):
    coeffs = I.random_sh_coeffs(8, nrhs, seed=seed)
    return I.sph_harm_combination(pts, coeffs, nrhs=nrhs) * A[None, :]


def _pair(torch, C, pts, kernel, n, theta, N0, W, **kw):
    """(persistent output, per-phase output, launches of each)."""
    out = []
    for nop in (False, True):
        P = C.plan_create(dev(torch, pts), kernel, n, theta, N0, precision=C.FP32_BULK,
                          max_nrhs=W.shape[0], no_persistent=nop, **kw)
        got = C.evaluate(P, dev(torch, W)).cpu().numpy()
        C.plan_sync(P)
        out.append((got, C.plan_stats(P)["launches_per_evaluate"]))
        C.plan_destroy(P)
    return out[0][0], out[1][0], out[0][1], out[1][1]


@pytest.mark.parametrize("kernel,nrhs", [(O.KERNEL_LAPLACE, 16), (O.KERNEL_NEWTON, 8),
                                         (O.KERNEL_SAL, 24), (O.KERNEL_BIHARMONIC, 32),
                                         (O.KERNEL_ONE, 8)])
def test_persistent_equals_per_phase_uniform(torch, C, kernel, nrhs):
    pts, A = I.cubed_sphere_grid(48)
    W = _weights(pts, A, nrhs, seed=kernel + 3)
    if kernel == O.KERNEL_ONE:
        W = W + A[None, :]
    per, phase, lp, lq = _pair(torch, C, pts, kernel, 8, 0.7, 64, W)
    assert lp < lq  # the persistent launch replaced the far, near, L2L and L2P launches
    assert np.array_equal(per, phase)


@pytest.mark.parametrize("name,mk,n,theta,N0", [
    ("random 20,000, n=6, N0=40 (P <= 128: two cells per far item)",
     lambda: I.random_sphere_points(20000, 71), 6, 0.7, 40),
    ("clustered caps, deep ragged tree, n=12, N0=30 (P > 128)",
     lambda: np.vstack([I.random_sphere_points(3000, 72),
                        (lambda v: v / np.linalg.norm(v, axis=1, keepdims=True))(
                            np.array([0.2, 0.5, 0.8]) + 0.02 * np.random.default_rng(73)
                            .standard_normal((4000, 3)))]), 12, 0.7, 30),
    ("50 points: every face is one leaf", lambda: I.random_sphere_points(50, 74), 4, 0.7, 100),
])
def test_persistent_equals_per_phase_ragged(torch, C, name, mk, n, theta, N0):
    pts = mk()
    W = np.random.default_rng(75).standard_normal((16, len(pts))) * (4 * math.pi / len(pts))
    per, phase, lp, lq = _pair(torch, C, pts, O.KERNEL_NEWTON, n, theta, N0, W)
    assert lp < lq
    assert np.array_equal(per, phase), name


def test_persistent_separate_targets_and_workspaces(torch, C):
    """Separate target points (outputs at the targets only) and two
    concurrent evaluations on their own workspaces and streams: the persistent
    launch equals the per-phase launches bit for bit."""
    src, tgt = I.random_sphere_points(12000, 76), I.random_sphere_points(3000, 77)
    W = np.random.default_rng(78).standard_normal((16, len(src))) / len(src)
    outs = []
    for nop in (False, True):
        P = C.plan_create_targets(dev(torch, src), dev(torch, tgt), C.KERNEL_NEWTON, 7, 0.7, 60,
                                  precision=C.FP32_BULK, max_nrhs=16, no_persistent=nop)
        outs.append(C.evaluate(P, dev(torch, W)).cpu().numpy())
        C.plan_sync(P)
        C.plan_destroy(P)
    assert outs[0].shape == (16, len(tgt), 1)
    assert np.array_equal(outs[0], outs[1])
    pts, A = I.cubed_sphere_grid(40)
    P = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, 7, 0.7, 50, precision=C.FP32_BULK,
                      max_nrhs=16)
    W1, W2 = dev(torch, _weights(pts, A, 16, seed=85)), dev(torch, _weights(pts, A, 16, seed=86))
    ref1 = C.evaluate(P, W1).cpu().numpy()
    ref2 = C.evaluate(P, W2).cpu().numpy()
    ws1, ws2 = C.workspace_create(P, 16), C.workspace_create(P, 16)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s1):
        o1 = C.evaluate_ws(P, ws1, W1, stream=s1.cuda_stream)
    with torch.cuda.stream(s2):
        o2 = C.evaluate_ws(P, ws2, W2, stream=s2.cuda_stream)
    torch.cuda.synchronize()
    C.plan_sync(P)
    assert np.array_equal(o1.cpu().numpy(), ref1) and np.array_equal(o2.cpu().numpy(), ref2)
    C.workspace_destroy(ws1)
    C.workspace_destroy(ws2)


def test_persistent_graph_replay_retargets_output(torch, C):
    pts, A = I.cubed_sphere_grid(40)
    plain = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, 7, 0.7, 50, precision=C.FP32_BULK,
                          max_nrhs=16)
    graph = C.plan_create(dev(torch, pts), C.KERNEL_LAPLACE, 7, 0.7, 50, precision=C.FP32_BULK,
                          max_nrhs=16, use_graphs=1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for call in range(3):
            W = dev(torch, _weights(pts, A, 16, seed=80 + call))
            ref = C.evaluate(plain, W, stream=s.cuda_stream)
            got = C.evaluate(graph, W, stream=s.cuda_stream)  # new buffers every call
            s.synchronize()
            assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy()), call
    C.plan_sync(graph, stream=s.cuda_stream)


def test_persistent_wait_timeout_is_reported_and_recoverable(torch, C):
    """A dependency that never completes (test hook): every wait gives up
    after its bound, the kernel returns, csfmm_plan_sync reports
    CSFMM_ERR_TIMEOUT once, and the same plan then evaluates correctly."""
    import time
    pts, A = I.cubed_sphere_grid(32)
    W = dev(torch, _weights(pts, A, 8, seed=90))
    P = C.plan_create(dev(torch, pts), C.KERNEL_NEWTON, 6, 0.7, 40, precision=C.FP32_BULK,
                      max_nrhs=8)
    ref = C.evaluate(P, W).cpu().numpy()
    C.plan_sync(P)
    C.plan_test_wait(P, True, limit_ms=50.0)
    t0 = time.perf_counter()
    C.evaluate(P, W)
    with pytest.raises(C.CsfmmError) as e:
        C.plan_sync(P)
    assert e.value.status == 5  # CSFMM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0  # one bound, not one per waiting item
    C.plan_test_wait(P, False, limit_ms=2000.0)
    got = C.evaluate(P, W).cpu().numpy()
    C.plan_sync(P)
    assert np.array_equal(got, ref)
    C.plan_destroy(P)
