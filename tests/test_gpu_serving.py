"""Serving loop on the GPU: continuous batching over resident plans.

Each request's result must be the same alone and in the mix (the kernels are
deterministic, the workspace private, the plan read-only), under slot and
memory pressure that forces queueing and plan eviction."""
import numpy as np
import pytest

from paper_2508_13550_gb300 import inputs as I
from gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = cuda_or_skip()
    from paper_2508_13550_gb300 import csfmm as C
    from paper_2508_13550_gb300 import serving as S
    return torch, C, S


def _alone(torch, C, S, grids, rec, precision):
    m, kid, deg = rec["m"], rec["kernel"], rec["degree"]
    plan = C.plan_create(grids.points(m), kid, deg, 0.7, S.leaf_size(deg), precision=precision,
                         max_nrhs=8)
    out = C.evaluate(plan, torch.from_numpy(rec["weights"]).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_results_same_alone_and_in_the_mix(env, precision):
    torch, C, S = env
    reqs = I.serving_requests(36, rate_hz=1e6, seed=11 + precision, ms=(8, 16, 24, 32),
                              nrhs_range=(1, 5), degree_range=(3, 7))
    grids = S.DeviceGrids((8, 16, 24, 32), "cuda")
    # a budget that holds only a few small plans: forces queueing and eviction
    server = C.Server(budget_bytes=24 << 20, slots=4)
    recs = S.run_stream(server, grids, reqs, rate_hz=None, precision=precision,
                        keep_outputs=True)
    st = server.stats()
    server.close()
    assert len(recs) == len(reqs) and all(r["status"] == 0 for r in recs)
    assert st["completed"] == len(reqs) and st["max_in_flight"] >= 2
    assert st["peak_bytes_held"] <= st["budget_bytes"]
    assert st["plans_evicted"] > 0
    for r in recs:
        alone = _alone(torch, C, S, grids, r, precision)
        assert np.array_equal(r["out"], alone), (r["id"], r["m"], r["kernel"])


def test_stream_with_arrivals_reports_latency(env):
    torch, C, S = env
    reqs = I.serving_requests(40, rate_hz=400.0, seed=3, ms=(16, 32, 64),
                              degree_range=(4, 8))
    grids = S.DeviceGrids((16, 32, 64), "cuda")
    server = C.Server(budget_bytes=2 << 30, slots=4)
    recs = S.run_stream(server, grids, reqs, rate_hz=400.0)
    server.close()
    summ = S.summarize(recs)
    assert summ["requests"] == 40 and summ["failed"] == 0
    assert 0 < summ["p50_ms"] <= summ["p99_ms"]
    assert all(r["admit_ms"] >= r["submit_ms"] and r["done_ms"] >= r["admit_ms"] for r in recs)


def test_requests_that_can_never_fit_are_refused(env):
    torch, C, S = env
    grids = S.DeviceGrids((64,), "cuda")
    server = C.Server(budget_bytes=1 << 20, slots=2)
    w = grids.weights(64, 1, 0)
    out = torch.empty((1, w.shape[1], 1), dtype=torch.float64, device="cuda")
    with pytest.raises(C.CsfmmError) as e:
        server.submit(grids.points(64), 64, 0, 8, 0.7, 256, 1, w, out)
    assert e.value.status == 3
    with pytest.raises(C.CsfmmError):
        server.submit(grids.points(64), 64, 0, 8, 0.7, 256, 1, w.repeat(9, 1), out)
    server.close()


@pytest.mark.parametrize("policy", ["fifo", "cheapest"])
def test_admission_order_policy(env, policy):
    """Three large requests (6 x 512^2 points) then ten small ones (6 x 16^2),
    all submitted at once, two slots.  First come first served starts the
    third large request before any small one; cheapest-first lets at most one
    large request run at a time and starts every small request before the
    third large one."""
    torch, C, S = env
    grids = S.DeviceGrids((16, 512), "cuda")
    pol = C.SERVE_FIFO if policy == "fifo" else C.SERVE_CHEAPEST_FIRST
    server = C.Server(budget_bytes=16 << 30, slots=2, policy=pol, age_ms=60000.0)
    # plans built before the burst, so that admissions are not held up by builds
    warm = [dict(id=i, arrival=0.0, m=m, kernel=0, nrhs=8, degree=d, seed=i)
            for i, (m, d) in enumerate(((512, 10), (16, 6)))]
    S.run_stream(server, grids, warm, rate_hz=None)
    burst = [(512, 8, 10, 10 + i) for i in range(3)] + [(16, 1, 6, 20 + i) for i in range(10)]
    bufs = []
    for m, nrhs, deg, seed in burst:  # every input ready before the first submission
        w = grids.weights(m, nrhs, seed)
        bufs.append((w, torch.empty((nrhs, w.shape[1], 1), dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    ids = [server.submit(grids.points(m), m, 0, deg, 0.7, S.leaf_size(deg), C.FP32_BULK, w, out)
           for (m, nrhs, deg, seed), (w, out) in zip(burst, bufs)]
    t = [server.wait(i) for i in ids]
    server.close()
    assert all(rc == 0 for rc, _ in t)
    admit = [tt["admit_ms"] for _, tt in t]
    third_large, small = admit[2], admit[3:]
    if policy == "fifo":
        assert third_large <= min(small)
    else:
        assert max(small) <= third_large
