"""Benchmark of the CSFMM evaluation pass on GB300.

Default workload (one step = one csfmm_evaluate of the whole hot path on a
resident plan): Newtonian kernel 1/sqrt(2(1 - x.y)) on the equiangular
cubed sphere with 6 x 1024^2 = 6,291,456 points, land-masked random weights,
degree n = 12, MAC 0.7, leaf size N0 = 576, FP32-bulk form, one right-hand
side.  Reported metric: FMM targets per second (N / time per evaluation),
with the relative l2 error against an FP64 direct sum on sampled targets.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank evaluates its own
replica of the workload on its GPU (the path has no data-path exchange:
replicas only); the time is the maximum over ranks and the value is the sum
of targets over ranks divided by it.  --impl reference times the CPU oracle
FMM (plain FP64 C) on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "newton-6m": dict(m=1024, kernel=2, n=12, theta=0.7, N0=576,
                      desc="Newtonian 1/sqrt(2(1-x.y)), cubed sphere 6x1024^2 = 6,291,456 "
                           "points, land-masked U[0,1] weights x cell area, n=12, MAC 0.7, "
                           "N0=576, 1 RHS"),
    "newton-1.5m": dict(m=512, kernel=2, n=12, theta=0.7, N0=576,
                        desc="Newtonian 1/sqrt(2(1-x.y)), cubed sphere 6x512^2 = 1,572,864 "
                             "points (profiling case of the same kernel shapes), n=12, MAC 0.7, "
                             "N0=576, 1 RHS"),
    "poisson-multirhs-1.5m": dict(m=512, kernel=0, n=10, theta=0.7, N0=400, nrhs=16,
                                  desc="Poisson log kernel, cubed sphere 6x512^2 = 1,572,864 "
                                       "points, 16 RHS of random Y_nm combinations, n=10, "
                                       "MAC 0.7, N0=400"),
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the FP32
# interaction kernels per kernel evaluation, from one ncu capture of the
# 6 x 512^2 Newtonian case (summarised under profiles/), valid only while the
# kernel sources (interact32.cu, fp32_math.cuh) hash to the given SHA-256
# prefix; the bench scales it to a launch by the evaluations the launch
# performs (the traffic of these kernels grows with the number of leaf pairs,
# cell pairs and points, as the evaluations do).
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2508_13550_gb300", "csrc", f)
                  for f in ("interact32.cu", "fp32_math.cuh")]
TRAFFIC_PER_EVAL = {
    "source_sha256": "a15ccee5df2fcfeb",
    "pp_sym_kernel": (35.367424e6 + 128.747264e6) / 6083051520,
    "near32x2_kernel": (236.443648e6 + 9.799936e6) / 3743870976,
    "far32x2_kernel": (40.254208e6 + 0.066048e6) / 615546672,
    "cc_sym_kernel": 6.239744e6 / 444180672,
}


def traffic_per_launch(kernel, evals):
    import hashlib
    h = hashlib.sha256()
    for path in KERNEL_SOURCES:
        with open(path, "rb") as f:
            h.update(f.read())
    sha = h.hexdigest()[:16]
    if sha != TRAFFIC_PER_EVAL["source_sha256"] or kernel not in TRAFFIC_PER_EVAL:
        return None
    return TRAFFIC_PER_EVAL[kernel] * evals


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, dist=None) -> float:
    """Maximum of x over the ranks of the default process group (x itself
    without one).  NCCL groups reduce on the current CUDA device, others on
    the CPU."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time
    (replicas: every rank processes the same number of units)."""
    return world * units_per_rank / seconds_max


def make_workload(name):
    from paper_2508_13550_gb300 import inputs as I
    wl = WORKLOADS[name]
    if name.startswith("newton"):
        pts, A, w = I.workload_newton_land(wl["m"])
    else:
        pts, A, w, _ = I.workload_multi_rhs(wl["m"], wl["nrhs"], with_exact=False)
    return wl, pts, A, np.ascontiguousarray(w)


def workload_config(args, wl, N, nrhs, world):
    """The `config` object of a bench line: the workload alone, identical for
    the library's arm and the reference arm of the same command."""
    return {"workload": args.workload, "desc": wl["desc"], "N": N, "nrhs": nrhs,
            "kernel": wl["kernel"], "degree": wl["n"], "theta": wl["theta"],
            "max_leaf": wl["N0"], "precision": args.precision,
            "parallelism": f"replicas x{world}"}


def cpu_oracle_sample(pts, w, wl, n_leaves, seed, repeats=1):
    """Times the CPU oracle FMM evaluation restricted to every target of
    n_leaves seeded random leaves (tree built beforehand, like a resident
    plan).  Returns (targets/s, seconds, targets, threads)."""
    import oracle as O
    f = O.FMM(pts, wl["n"], wl["theta"], wl["N0"])
    C = f.cells()
    leaf = np.where(C["child"].max(axis=1) < 0)[0]
    rng = np.random.default_rng(seed)
    pick = rng.choice(leaf, min(n_leaves, len(leaf)), replace=False)
    order = f.order()
    tg = np.concatenate([order[C["begin"][c]:C["end"][c]] for c in pick])
    t0 = time.perf_counter()
    for _ in range(repeats):
        f.evaluate(wl["kernel"], w, tg)
    dt = (time.perf_counter() - t0) / repeats
    rate, threads = len(tg) / dt, O.num_threads()
    # one thread on the first sixteenth of the leaves
    tg1 = np.concatenate([order[C["begin"][c]:C["end"][c]] for c in pick[:max(1, len(pick) // 16)]])
    O.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        f.evaluate(wl["kernel"], w, tg1)
        dt1 = time.perf_counter() - t0
    finally:
        O.set_num_threads(threads)
    return rate, dt, len(tg), threads, (len(tg1) / dt1, dt1, len(tg1))


def fp64_at_matched_accuracy(Cs, torch, dpts, dw, wl, dim, dtg, ds, err32, ms32_per_rhs):
    """The plain single-RHS FP64 GPU FMM at the accuracy of the FP32-bulk
    form: the smallest degree n' (N0 = 4 n'^2, same MAC) whose error against
    the FP64 direct sum on the same sampled targets is at most err32, timed
    with CUDA events.  Returns the degrees tried and the speedup of the
    FP32-bulk evaluation over that FP64 evaluation."""
    dev = dpts.device
    stream = torch.cuda.current_stream(dev)
    tried = []
    for n in range(4, wl["n"] + 1):
        p = Cs.plan_create(dpts, wl["kernel"], n, wl["theta"], 4 * n * n, precision=Cs.FP64,
                           max_nrhs=1)
        o = torch.empty((1, dpts.shape[0], dim), dtype=torch.float64, device=dev)
        Cs.evaluate(p, dw[:1], out=o)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Cs.evaluate(p, dw[:1], out=o)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e = float(torch.linalg.norm(o[:1, dtg] - ds) / torch.linalg.norm(ds))
        ms = e0.elapsed_time(e1)
        Cs.plan_destroy(p)
        del o
        tried.append({"degree": n, "max_leaf": 4 * n * n, "rel_err_vs_fp64_ds": e,
                      "ms_per_eval_1rhs": ms})
        if e <= err32:
            return {"degree": n, "ms_per_eval_1rhs": ms, "rel_err_vs_fp64_ds": e,
                    "fp32_bulk_rel_err": err32,
                    "speedup_of_fp32_bulk_per_rhs": ms / ms32_per_rhs, "tried": tried}
    return {"degree": None, "fp32_bulk_rel_err": err32, "tried": tried,
            "note": "no FP64 degree up to the workload's reaches the FP32-bulk error"}


def timed_steps(torch, Cs, plan, dw, out, stream, steps):
    """CUDA-event time of each of `steps` evaluations (ms), synchronised."""
    res = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Cs.evaluate(plan, dw, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        res.append(e0.elapsed_time(e1))
    return res


def side_workloads(args, torch, Cs, n_sm, sm_max):
    """The other benchmark workloads measured in the same run, each on its
    own plan with inputs resident (CUDA events, median of the steps):
    Biot-Savart on 6 x 256^2 points (n = 10, FP64 and FP32 bulk) and the
    16-right-hand-side Poisson workload on 6 x 512^2 points (n = 10, FP32
    bulk, persistent launch).  Errors against the FP64 direct sum on sampled
    targets."""
    from paper_2508_13550_gb300 import inputs as I
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    res = {}
    rng = np.random.default_rng(20250814)

    def case(pts, w, kid, n, N0, prec, nrhs, samples):
        dp = torch.from_numpy(pts).to(dev)
        dw = torch.from_numpy(np.ascontiguousarray(w)).to(dev)
        dim = Cs.kernel_dim(kid)
        tg = torch.from_numpy(np.sort(rng.choice(len(pts), samples, replace=False))
                              .astype(np.int64)).to(dev)
        ds = Cs.direct(dp, kid, dw, precision=Cs.FP64, targets=tg)
        plan = Cs.plan_create(dp, kid, n, 0.7, N0, precision=prec, max_nrhs=nrhs)
        out = torch.empty((nrhs, len(pts), dim), dtype=torch.float64, device=dev)
        for _ in range(3):
            Cs.evaluate(plan, dw, out=out)
        torch.cuda.synchronize()
        steps = timed_steps(torch, Cs, plan, dw, out, stream, args.side_steps)
        Cs.plan_enable_timing(plan, True)
        Cs.evaluate(plan, dw, out=out)
        ph, calls = Cs.plan_phase_times(plan)
        Cs.plan_enable_timing(plan, False)
        Cs.plan_sync(plan)
        st = Cs.plan_stats(plan)
        d = out[:, tg] - ds
        errs = [float(torch.linalg.norm(d[r]) / torch.linalg.norm(ds[r])) for r in range(nrhs)]
        ms = statistics.median(steps)
        Cs.plan_destroy(plan)
        return {"N": len(pts), "nrhs": nrhs, "degree": n, "max_leaf": N0,
                "precision": "fp32" if prec == Cs.FP32_BULK else "fp64",
                "ms_per_eval": ms, "step_ms_min": min(steps), "steps": len(steps),
                "targets_per_s": len(pts) * nrhs / (ms / 1e3),
                "kernel_evals_per_s": sum(st["evals"]) / (ms / 1e3),
                "rel_err_vs_fp64_ds_max_over_rhs": max(errs), "err_samples": samples,
                "phase_ms": {k: v / max(calls, 1) for k, v in ph.items()},
                "launches_per_evaluate": st["launches_per_evaluate"]}

    pts, A, w, _ = I.workload_rh_biot_savart(256)
    res["biot_savart_393k"] = {
        "desc": "Biot-Savart, RH wave-4 vorticity + 1e-3 noise, cubed sphere 6x256^2 = 393,216 "
                "points, n=10, MAC 0.7, N0=400",
        "fp64": case(pts, w, Cs.KERNEL_BIOT_SAVART, 10, 400, Cs.FP64, 1, 512),
        "fp32_bulk": case(pts, w, Cs.KERNEL_BIOT_SAVART, 10, 400, Cs.FP32_BULK, 1, 512)}
    pts, A, W, _ = I.workload_multi_rhs(512, 16, with_exact=False)
    mr = case(pts, W, Cs.KERNEL_LAPLACE, 10, 400, Cs.FP32_BULK, 16, 256)
    ms_k = mr["phase_ms"].get("near", 0.0)
    per_clk = 128.0 / (6 + 16)
    mr["roofline"] = {"kernel": "persistent_kernel (CC, CP, PP, PC for 16 RHS, L2L, L2P)",
                      "bound": "alu (FP32 pipe: 6 + 16 lane-ops per evaluation)",
                      "achieved_geval_per_s": mr["kernel_evals_per_s"] / 1e9 if ms_k else None,
                      "kernel_ms": ms_k,
                      "kernel_geval_per_s": (mr["kernel_evals_per_s"] * mr["ms_per_eval"] / ms_k
                                             / 1e9) if ms_k else None,
                      "peak_geval_per_s": n_sm * per_clk * sm_max / 1e3,
                      "frac": (mr["kernel_evals_per_s"] * mr["ms_per_eval"] / ms_k)
                              / (n_sm * per_clk * sm_max * 1e6) if ms_k else None}
    res["poisson_16rhs_1.5m"] = dict(
        desc="Poisson log kernel, 16 RHS of random Y_nm combinations (n <= 32), cubed sphere "
             "6x512^2 = 1,572,864 points, n=10, MAC 0.7, N0=400, FP32 bulk", **mr)
    return res


def run_reference(args):
    """CPU oracle arm: each step evaluates a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    wl, pts, A, w = make_workload(args.workload)
    f = O.FMM(pts, wl["n"], wl["theta"], wl["N0"])
    C = f.cells()
    leaf = np.where(C["child"].max(axis=1) < 0)[0]
    order = f.order()
    rng = np.random.default_rng(7)
    per_step = args.ref_leaves

    def step():
        pick = rng.choice(leaf, per_step, replace=False)
        tg = np.concatenate([order[C["begin"][c]:C["end"][c]] for c in pick])
        f.evaluate(wl["kernel"], w[:1], tg)
        return len(tg)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    nt = 0
    for _ in range(args.steps):
        nt += step()
    dt = time.perf_counter() - t0
    val = nt / dt
    sample = (f"per step: all targets of {per_step} seeded random leaves "
              f"({nt // max(args.steps, 1)} targets) of the {wl['desc']} workload; "
              f"tree built once before timing")
    line = {"impl": "reference", "metric": "FMM targets/s at N=6.3M", "value": val,
            "unit": "targets/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(args, wl, len(pts), w.shape[0], args.gpus),
            "cpu_baseline": {"value": val, "unit": "targets/s", "cores": O.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "targets/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2508_13550_gb300 import csfmm as Cs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl, pts, A, w = make_workload(args.workload)
    wl_base = wl
    N = len(pts)
    nrhs = w.shape[0]
    prec = Cs.FP32_BULK if args.precision == "fp32" else Cs.FP64
    dpts = torch.from_numpy(pts).to(dev)
    dw = torch.from_numpy(w).to(dev)
    tuned = None
    if nrhs > 1 and args.autotune and prec == Cs.FP32_BULK:
        # leaf size and right-hand-side chunk picked by the library's autotuner
        # (timed evaluations, error within 2x of the default's), before timing
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            tuned = Cs.autotune(dpts, wl["kernel"], wl["n"], wl["theta"], dw, precision=prec,
                                cache_path=os.path.join(td, "tune.txt"))
        wl = dict(wl, N0=tuned["max_leaf"])
        log("autotune", tuned)
    plan = Cs.plan_create(dpts, wl["kernel"], wl["n"], wl["theta"], wl["N0"], precision=prec,
                          max_nrhs=max(nrhs, 1),
                          rhs_chunk=tuned["rhs_chunk"] if tuned else 0,
                          no_persistent=args.no_persistent, schedule=args.schedule)
    st = Cs.plan_stats(plan)
    dim = Cs.kernel_dim(wl["kernel"])
    out = torch.empty((nrhs, N, dim), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        Cs.evaluate(plan, dw, out=out)
    torch.cuda.synchronize(dev)
    Cs.plan_sync(plan)

    # timed region (inputs resident; working set >> 129 MB L2)
    Cs.plan_enable_timing(plan, True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for _ in range(args.steps):
            Cs.evaluate(plan, dw, out=out)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
    Cs.plan_enable_timing(plan, False)
    ms = ev0.elapsed_time(ev1)
    phases, calls = Cs.plan_phase_times(plan)
    Cs.plan_sync(plan)
    # per-step times (after the timed region): median and minimum of K steps
    step_ms = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Cs.evaluate(plan, dw, out=out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        step_ms.append(e0.elapsed_time(e1))
    launches = Cs.plan_stats(plan)["launches_per_evaluate"] * args.steps
    ms = max_over_ranks(ms, dist)
    ms_step = ms / args.steps
    value = whole_job_rate(N * nrhs, world, ms_step / 1e3)

    # end to end through the host-buffer entry point: H2D weights, evaluate, D2H result
    hw = torch.from_numpy(w).pin_memory()
    hout = torch.empty((nrhs, N, dim), dtype=torch.float64).pin_memory()
    lib = Cs.load()
    import ctypes
    for _ in range(2):
        Cs._check(lib.csfmm_evaluate_host(plan.handle, ctypes.c_void_p(hw.data_ptr()), nrhs,
                                          ctypes.c_void_p(hout.data_ptr()),
                                          ctypes.c_void_p(stream.cuda_stream)))
    e2e_steps = max(3, min(args.steps, 10))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Cs._check(lib.csfmm_evaluate_host(plan.handle, ctypes.c_void_p(hw.data_ptr()), nrhs,
                                          ctypes.c_void_p(hout.data_ptr()),
                                          ctypes.c_void_p(stream.cuda_stream)))
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist)
    e2e_val = whole_job_rate(N * nrhs, world, e2e_s)

    # accuracy against the FP64 direct sum on sampled targets (GPU direct sum)
    rng = np.random.default_rng(20250813)
    tg = np.sort(rng.choice(N, args.err_samples, replace=False)).astype(np.int64)
    dtg = torch.from_numpy(tg).to(dev)
    ds = Cs.direct(dpts, wl["kernel"], dw[:1], precision=Cs.FP64, targets=dtg)
    got = out[:1, dtg]
    err = float(torch.linalg.norm(got - ds) / torch.linalg.norm(ds))

    # the plain single-RHS FP64 GPU FMM on the same workload, for the speedup
    fp64 = None
    fp64_matched = None
    if args.fp64_compare and prec == Cs.FP32_BULK:
        p64 = Cs.plan_create(dpts, wl["kernel"], wl["n"], wl["theta"], wl["N0"],
                             precision=Cs.FP64, max_nrhs=1)
        o64 = torch.empty((1, N, dim), dtype=torch.float64, device=dev)
        Cs.evaluate(p64, dw[:1], out=o64)  # warm-up
        torch.cuda.synchronize(dev)
        steps64 = timed_steps(torch, Cs, p64, dw[:1], o64, stream, args.fp64_steps)
        ms64 = sum(steps64) / len(steps64)
        err64 = float(torch.linalg.norm(o64[:1, dtg] - ds) / torch.linalg.norm(ds))
        st64 = Cs.plan_stats(p64)
        fp64 = {"ms_per_eval_1rhs": ms64, "steps": len(steps64), "step_ms_min": min(steps64),
                "step_ms_max": max(steps64), "rel_err_vs_fp64_ds": err64,
                "kernel_evals_per_s": sum(st64["evals"]) / (ms64 / 1e3),
                "speedup_of_fp32_bulk_per_rhs": ms64 / (ms_step / nrhs)}
        Cs.plan_destroy(p64)
        del o64
        fp64_matched = fp64_at_matched_accuracy(Cs, torch, dpts, dw, wl, dim, dtg, ds, err,
                                                ms_step / nrhs)

    peaks, peak_kind = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # ALU roofline of the interaction kernels, in kernel evaluations (one
    # K(x, y) per target-source pair, shared by all right-hand sides):
    #  - one right-hand side: 7 FP32-pipe operations and one MUFU operation
    #    (rsqrt / lg2 / rcp) per evaluation; a GB300 SM has 128 FP32 lanes and
    #    16 MUFU lanes per clock, so the MUFU pipe bounds at 16/clock/SM;
    #  - nrhs = 8 or 16 (multi32_kernel): 6 FP32 operations for |r|^2 plus
    #    one FMA per right-hand side, so the FP32 pipe bounds at
    #    128 / (6 + nrhs) evaluations/clock/SM.
    if nrhs == 1:
        per_sm_clk = {2: 16.0, 0: 16.0, 1: 128.0 / 11.0, 100: 128.0 / 4.0}[wl["kernel"]]
    else:
        per_sm_clk = min(16.0, 128.0 / (6 + min(nrhs, 16)))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_evals = n_sm * per_sm_clk * sm_max * 1e6
    ncalls = max(calls, 1)
    ev_sym = st.get("sym_evals", 0) if nrhs == 1 else 0
    # mirrored CC cell pairs: P^2 kernel values each, serving two CC entries
    ev_cc = st.get("cc_sym_pairs", 0) * (wl["n"] + 1) ** 4 if nrhs == 1 else 0
    if nrhs == 1:
        kern = {
            # kernel: (kernel evaluations per launch, ms per launch)
            "pp_sym_kernel": (ev_sym, phases.get("ppsym", 0.0) / ncalls),
            "near32x2_kernel": (st["evals"][0] + st["evals"][1] - 2 * ev_sym, phases["near"] / ncalls),
            "far32x2_kernel": (st["evals"][2] + st["evals"][3] - 2 * ev_cc, phases["far"] / ncalls),
        }
        what = {"pp_sym_kernel": "sym_kernel on mirrored PP leaf pairs, one evaluation per pair",
                "near32x2_kernel": "self and unmirrored PP, PC",
                "far32x2_kernel": "CP and unmirrored CC"}
        if ev_cc > 0:
            kern["cc_sym_kernel"] = (ev_cc, phases.get("ccsym", 0.0) / ncalls)
            what["cc_sym_kernel"] = "sym_kernel on mirrored CC cell pairs, one evaluation per pair"
    elif phases.get("far", 0.0) == 0.0:
        # the persistent launch: far field, near field, L2L and L2P of all
        # right-hand sides in one kernel (its time is the NEAR phase)
        kern = {"persistent_kernel": (sum(st["evals"]), phases["near"] / ncalls)}
        what = {"persistent_kernel": f"CC, CP, PP, PC, L2L, L2P for {nrhs} right-hand sides "
                                     "in one launch"}
    else:
        # per evaluation of all right-hand sides (chunks of 16 in one launch)
        kern = {
            "multi32_kernel (near)": (st["evals"][0] + st["evals"][1], phases["near"] / ncalls),
            "multi32_kernel (far)": (st["evals"][2] + st["evals"][3], phases["far"] / ncalls),
        }
        what = {"multi32_kernel (near)": f"PP, PC for {nrhs} right-hand sides",
                "multi32_kernel (far)": f"CC, CP for {nrhs} right-hand sides"}
    dom = max(kern, key=lambda k: kern[k][1])
    dom_evals, dom_ms = kern[dom]
    achieved = dom_evals / (dom_ms / 1e3)
    traffic = traffic_per_launch(dom, dom_evals) if nrhs == 1 else None
    line = {
        "metric": "FMM targets/s at N=6.3M" if N == 6291456 else f"FMM targets/s at N={N}",
        "value": value, "unit": "targets/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == Cs.FP32_BULK else "f64", "data": "synthetic",
        "autotuned": tuned,
        "schedule": args.schedule,
        "config": workload_config(args, wl_base, N, nrhs, world),
        "l2": "inputs larger than L2 (plan + workspace "
              f"{st['device_bytes'] / 1e9:.2f} GB resident)",
        "rel_err_vs_fp64_ds": err, "err_samples": args.err_samples,
        # a mirrored pair's kernel value serves two interactions
        "kernel_evals_per_s": world * (sum(st["evals"]) - ev_sym - ev_cc) / (ms_step / 1e3),
        "interactions_per_s": world * sum(st["evals"]) * nrhs / (ms_step / 1e3),
        "phase_ms": {k: v / max(calls, 1) for k, v in phases.items()},
        "plan_build_ms": st["build_ms"],
        "fp64_gpu_fmm": fp64,
        "fp64_gpu_fmm_at_matched_accuracy": fp64_matched,
        "gpu_launches": launches,
        "e2e": {"value": e2e_val, "unit": "targets/s",
                "h2d_bytes_per_step": int(w.nbytes), "d2h_bytes_per_step": int(8 * nrhs * N * dim)},
        "roofline": {"kernel": f"{dom} ({what[dom]})", "bound": "alu",
                     "achieved": achieved / 1e9, "peak": peak_evals / 1e9, "unit": "Geval/s",
                     "frac": achieved / peak_evals,
                     "traffic": traffic, "traffic_unit": "bytes per launch",
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the "
                                       "6 x 512^2 case, scaled by evaluations per launch"
                                       if traffic is not None else None,
                     "peak_source": f"{peak_kind} sm_max_mhz x {n_sm} SMs (device "
                                    f"attribute) x {per_sm_clk:.2f} evals/clk/SM",
                     "sm_count": n_sm},
        "kernels": {k: {"evals_per_launch": e, "ms_per_launch": m,
                        "geval_per_s": (e / (m / 1e3) / 1e9) if m > 0 else None,
                        "frac_of_alu_peak": (e / (m / 1e3) / peak_evals) if m > 0 else None}
                    for k, (e, m) in kern.items()},
        "clocks": clk.summary(),
        "step_ms": {"median": statistics.median(step_ms), "min": min(step_ms),
                    "n": len(step_ms)},
    }
    if rank == 0 and world == 1 and nrhs == 1 and prec == Cs.FP32_BULK:
        # every phase alone on one stream (CSFMM_SCHED_NO_OVERLAP), so that each
        # interaction kernel's event time is its own, not shared with the side
        # stream's far field
        p1 = Cs.plan_create(dpts, wl["kernel"], wl["n"], wl["theta"], wl["N0"], precision=prec,
                            max_nrhs=1, schedule=Cs.SCHED_NO_OVERLAP)
        first = Cs.plan_stats(p1)["build_ms"]
        Cs.plan_destroy(p1)  # its memory stays in the library's pool for the rebuild
        p1 = Cs.plan_create(dpts, wl["kernel"], wl["n"], wl["theta"], wl["N0"], precision=prec,
                            max_nrhs=1, schedule=Cs.SCHED_NO_OVERLAP)
        line["plan_build_ms_warm_pool"] = Cs.plan_stats(p1)["build_ms"]
        line["plan_build_ms_second_plan"] = first
        for _ in range(2):
            Cs.evaluate(p1, dw, out=out)
        Cs.plan_enable_timing(p1, True)
        for _ in range(5):
            Cs.evaluate(p1, dw, out=out)
        torch.cuda.synchronize(dev)
        ph1, c1 = Cs.plan_phase_times(p1)
        Cs.plan_enable_timing(p1, False)
        Cs.plan_destroy(p1)
        alone = {}
        for k, (e, _) in kern.items():
            phase = {"pp_sym_kernel": "ppsym", "near32x2_kernel": "near",
                     "far32x2_kernel": "far", "cc_sym_kernel": "ccsym"}[k]
            m = ph1[phase] / max(c1, 1)
            alone[k] = {"ms_per_launch": m, "geval_per_s": e / (m / 1e3) / 1e9,
                        "frac_of_alu_peak": e / (m / 1e3) / peak_evals}
        line["kernels_alone"] = alone
        line["phase_ms_alone"] = {k: v / max(c1, 1) for k, v in ph1.items()}
        line["kernels_alone_note"] = ("5 evaluations with every phase on one stream "
                                      "(CSFMM_SCHED_NO_OVERLAP), CUDA events per phase; "
                                      "plan_build_ms_warm_pool: a rebuild of that plan "
                                      "after destroying it, its memory reused from the "
                                      "library's pool")
    if rank == 0 and world == 1 and args.side_workloads:
        line["other_workloads"] = side_workloads(args, torch, Cs, n_sm, sm_max)
    if rank == 0 and world == 1 and args.serve_sample > 0:
        line["serving"] = run_serving(args, sample=args.serve_sample)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, ntg, cores, one = cpu_oracle_sample(pts, w[:1], wl, args.cpu_leaves, 3)
        line["cpu_baseline"] = {"value": v, "unit": "targets/s", "cores": cores, "kind": "oracle",
                                "sample": f"all {ntg} targets of {args.cpu_leaves} seeded random "
                                          f"leaves, FP64 oracle FMM, {dt:.1f} s",
                                "single_thread": {"value": one[0], "unit": "targets/s",
                                                  "sample": f"{one[2]} targets, {one[1]:.1f} s"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    Cs.plan_destroy(plan)
    if dist:
        dist.destroy_process_group()
    return 0


def run_serving(args, sample=None):
    """Serving stream (seeded requests: m ~ U{64..1024}, kernel ~ U{Laplace,
    Biot-Savart, Newtonian}, 1-8 RHS, degree 8-12, FP32 bulk, N0 = 4 n^2):
    warm-up requests fill the plan cache, a burst measures the saturation
    request rate, then the stream runs with Poisson arrivals at 70% of it.
    Returns the summary dict."""
    import torch
    from paper_2508_13550_gb300 import csfmm as Cs
    from paper_2508_13550_gb300 import inputs as I
    from paper_2508_13550_gb300 import serving as S
    n_req = sample or args.serve_requests
    ms = (64, 128, 256, 512, 1024)
    grids = S.DeviceGrids(ms, torch.device("cuda", torch.cuda.current_device()))
    policy = Cs.SERVE_FIFO if args.serve_policy == "fifo" else Cs.SERVE_CHEAPEST_FIRST
    server = Cs.Server(budget_bytes=int(args.serve_budget_gb * (1 << 30)), slots=args.serve_slots,
                       policy=policy, age_ms=args.serve_age_ms)
    warm = I.serving_requests(120, rate_hz=1e6, seed=I.MASTER_SEED + 50)
    S.run_stream(server, grids, warm, rate_hz=None)
    burst = I.serving_requests(min(200, n_req), rate_hz=1e6, seed=I.MASTER_SEED + 51)
    sat = S.summarize(S.run_stream(server, grids, burst, rate_hz=None))
    rate = 0.7 * sat["requests_per_s"]
    reqs = I.serving_requests(n_req, rate_hz=rate, seed=I.MASTER_SEED + 5)
    recs = S.run_stream(server, grids, reqs, rate_hz=rate)
    summ = S.summarize(recs)
    st = server.stats()
    server.close()
    summ.update({"arrival_rate_hz": rate, "saturation_requests_per_s": sat["requests_per_s"],
                 "saturation_targets_per_s": sat["targets_per_s"], "slots": args.serve_slots,
                 "budget_gb": args.serve_budget_gb, "plans_built": st["plans_built"],
                 "policy": args.serve_policy, "age_ms": args.serve_age_ms,
                 "plans_evicted": st["plans_evicted"],
                 "peak_bytes_held_gb": st["peak_bytes_held"] / 2 ** 30,
                 "max_in_flight": st["max_in_flight"]})
    return summ


def run_accuracy_sweep(args):
    """E(FS64, DS) (FMM truncation) and E(FS32, DS) (FP32-bulk form) against
    an FP64 GPU direct sum on sampled targets (MAC 0.7, N0 = 4 n^2):
    land-masked Newtonian field on the cubed sphere with m = args.sweep_m and
    the Y43 Poisson field with m = args.sweep_m / 2, for the degrees in
    args.sweep_degrees; then the 16-RHS Poisson workload (m = 512, n = 10)
    over all right-hand sides."""
    import torch
    from paper_2508_13550_gb300 import csfmm as Cs
    from paper_2508_13550_gb300 import inputs as I
    rows = []
    degrees = [int(x) for x in args.sweep_degrees.split(",")]

    def errors(dp, kid, dw, tg, ds, n, N0, nrhs):
        row = {}
        for key, prec in (("E64", Cs.FP64), ("E32", Cs.FP32_BULK)):
            P = Cs.plan_create(dp, kid, n, 0.7, N0, precision=prec, max_nrhs=nrhs)
            out = Cs.evaluate(P, dw)
            torch.cuda.synchronize()
            d = out[:, tg] - ds
            row[key] = float(torch.linalg.norm(d) / torch.linalg.norm(ds))
            row[key + "_bias"] = float(d.sum() / ds.abs().sum())
            Cs.plan_destroy(P)
        row["E32_over_E64"] = row["E32"] / row["E64"]
        return row

    def sample(N, seed=20250813):
        rng = np.random.default_rng(seed)
        return torch.from_numpy(np.sort(rng.choice(N, args.err_samples, replace=False))
                                .astype(np.int64)).cuda()

    for name, kid, m in (("newton", Cs.KERNEL_NEWTON, args.sweep_m),
                         ("laplace_y43", Cs.KERNEL_LAPLACE, args.sweep_m // 2)):
        pts, A = I.cubed_sphere_grid(m)
        w = (I.land_mask_field(pts, I.MASTER_SEED + 3) if name == "newton"
             else I.real_sph_harm(4, 3, pts)) * A
        dp = torch.from_numpy(pts).cuda()
        dw = torch.from_numpy(w[None].copy()).cuda()
        tg = sample(len(pts))
        ds = Cs.direct(dp, kid, dw, precision=Cs.FP64, targets=tg)
        for n in degrees:
            row = {"field": name, "m": m, "N": len(pts), "n": n, "N0": 4 * n * n}
            row.update(errors(dp, kid, dw, tg, ds, n, 4 * n * n, 1))
            rows.append(row)
            log(row)
    pts, A, w, _ = I.workload_multi_rhs(512, 16, with_exact=False)
    dp = torch.from_numpy(pts).cuda()
    dw = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    tg = sample(len(pts))
    ds = Cs.direct(dp, Cs.KERNEL_LAPLACE, dw, precision=Cs.FP64, targets=tg)
    row = {"field": "poisson_16rhs", "m": 512, "N": len(pts), "n": 10, "N0": 400}
    row.update(errors(dp, Cs.KERNEL_LAPLACE, dw, tg, ds, 10, 400, 16))
    rows.append(row)
    log(row)
    return {"metric": "FMM rel err vs FP64 direct sum (degree sweep)", "unit": "rel l2",
            "config": {"workload": "accuracy-sweep", "theta": 0.7,
                       "err_samples": args.err_samples}, "rows": rows}


def run_cstc_vs_fmm(args):
    """Runtime of the tree code against the CSFMM and the direct sum on the
    GPU (the paper's serial runtime comparison: Laplace kernel, MAC 0.7,
    degree 6): Poisson Y43 field on 6 x m^2 cubed-sphere points, N0 = 4 n^2.
    Each fast sum is timed with CUDA events after a warm-up evaluation; the
    FP32 direct sum covers all N^2 pairs, the FP64 direct sum a sample of
    targets scaled to N.  Errors are against the FP64 direct sum on sampled
    targets."""
    import torch
    from paper_2508_13550_gb300 import csfmm as Cs
    from paper_2508_13550_gb300 import inputs as I
    m, n, theta = args.sweep_m, 6, 0.7
    pts, A, w, _ = I.workload_poisson_y43(m)
    N = len(pts)
    dp = torch.from_numpy(pts).cuda()
    dw = torch.from_numpy(w).cuda()
    rng = np.random.default_rng(20250813)
    tg = torch.from_numpy(np.sort(rng.choice(N, args.err_samples, replace=False))
                          .astype(np.int64)).cuda()

    def timed(fn, reps=1):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    ms_ds64_sample, ds = timed(lambda: Cs.direct(dp, Cs.KERNEL_LAPLACE, dw, precision=Cs.FP64,
                                                   targets=tg))
    rows = {"direct FP64 (scaled from the sample)": {"ms": ms_ds64_sample * N / len(tg)}}
    ms_ds32, o = timed(lambda: Cs.direct(dp, Cs.KERNEL_LAPLACE, dw, precision=Cs.FP32_BULK))
    rows["direct FP32 (all pairs)"] = {"ms": ms_ds32, "rel_err": float(
        torch.linalg.norm(o[:, tg] - ds) / torch.linalg.norm(ds))}
    for name, prec in (("FP64", Cs.FP64), ("FP32", Cs.FP32_BULK)):
        P = Cs.plan_create(dp, Cs.KERNEL_LAPLACE, n, theta, 4 * n * n, precision=prec)
        for meth, fn in (("CSFMM", Cs.evaluate), ("CSTC", Cs.evaluate_cstc)):
            ms, o = timed(lambda: fn(P, dw), reps=3)
            rows[f"{meth} {name}"] = {"ms": ms, "rel_err": float(
                torch.linalg.norm(o[:, tg] - ds) / torch.linalg.norm(ds))}
            log(meth, name, rows[f"{meth} {name}"])
        Cs.plan_destroy(P)
    ratios = {
        "CSTC_FP64_over_CSFMM_FP64": rows["CSTC FP64"]["ms"] / rows["CSFMM FP64"]["ms"],
        "direct_FP64_over_CSTC_FP64": rows["direct FP64 (scaled from the sample)"]["ms"]
                                      / rows["CSTC FP64"]["ms"],
        "CSTC_FP32_over_CSFMM_FP32": rows["CSTC FP32"]["ms"] / rows["CSFMM FP32"]["ms"],
        "direct_FP32_over_CSTC_FP32": rows["direct FP32 (all pairs)"]["ms"]
                                      / rows["CSTC FP32"]["ms"],
    }
    return {"metric": "runtime of direct sum, CSTC and CSFMM (Laplace, MAC 0.7, n = 6)",
            "unit": "ms", "config": {"workload": "cstc-vs-fmm", "m": m, "N": N, "degree": n,
                                     "theta": theta, "max_leaf": 4 * n * n,
                                     "err_samples": args.err_samples},
            "rows": rows, "ratios": ratios,
            "paper_context": "serial CPU, icosahedral N = 2,621,442: CSTC 25x faster than the "
                             "direct sum, CSFMM 30x faster than CSTC"}


def run_paper_table(args):
    """Table "csfmmerrors" of the paper on the GPU: CSFMM approximation error
    E(phi_FS, phi_DS) (normalised by phi_EX, area-weighted, Sec. 10.2) for the
    Poisson problem with Y00, Y43 and Y85 on the icosahedral grid (level 8:
    N = 655362), MAC 0.5 / 0.7 / 0.9, degree n = 2:2:14, N0 = 4 n^2, FP64
    form; the three fields are the three right-hand sides of one evaluation
    and the FP64 direct sum is taken on sampled targets.  Prints each entry
    beside the paper's (tests/golden/csfmm_errors_table.txt)."""
    import torch
    from paper_2508_13550_gb300 import csfmm as Cs
    from paper_2508_13550_gb300 import inputs as I
    pts, A = I.icosahedral_grid(args.ico_level)
    N = len(pts)
    Y = np.stack([I.real_sph_harm(0, 0, pts), I.real_sph_harm(4, 3, pts),
                  I.real_sph_harm(8, 5, pts)])
    # exact potentials: Funk-Hecke eigenvalues 1/(n(n+1)) and, for n = 0,
    # int G_L dS = 1 - ln 2 (Eqs. G_L_1, G_L_2)
    EX = np.stack([(1.0 - math.log(2.0)) * Y[0], Y[1] / 20.0, Y[2] / 72.0])
    W = np.ascontiguousarray(Y * A)
    dp = torch.from_numpy(pts).cuda()
    dW = torch.from_numpy(W).cuda()
    rng = np.random.default_rng(20250813)
    tg = np.sort(rng.choice(N, min(args.err_samples, N), replace=False)).astype(np.int64)
    dtg = torch.from_numpy(tg).cuda()
    ds = Cs.direct(dp, Cs.KERNEL_LAPLACE, dW, precision=Cs.FP64, targets=dtg)[:, :, 0].cpu().numpy()
    At = A[tg]
    den = np.sum(EX[:, tg] ** 2 * At, axis=1)
    e_ds = np.sqrt(np.sum((ds - EX[:, tg]) ** 2 * At, axis=1) / den)
    paper = {}
    with open(os.path.join(ROOT, "tests", "golden", "csfmm_errors_table.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                paper[(line[0], float(line[1]))] = [float(x) for x in line[2:]]
    rows = []
    names = ("Y00", "Y43", "Y85")
    for mac in (0.9, 0.7, 0.5):
        for n in range(2, 15, 2):
            P = Cs.plan_create(dp, Cs.KERNEL_LAPLACE, n, mac, 4 * n * n, precision=Cs.FP64,
                               max_nrhs=3)
            out = Cs.evaluate(P, dW)
            torch.cuda.synchronize()
            fs = out[:, dtg, 0].cpu().numpy()
            Cs.plan_destroy(P)
            e = np.sqrt(np.sum((fs - ds) ** 2 * At, axis=1) / den)
            for k, nm in enumerate(names):
                ref = paper[(nm, mac)][n // 2 - 1]
                rows.append({"field": nm, "mac": mac, "n": n, "E_FS_DS": float(e[k]),
                             "paper": ref, "ratio": float(e[k]) / ref})
            log(mac, n, [f"{x:.2e}" for x in e])
    ratios = np.array([r["ratio"] for r in rows])
    return {"metric": "CSFMM approximation error E(phi_FS, phi_DS) vs Table csfmmerrors",
            "unit": "rel l2 (normalised by phi_EX)",
            "config": {"workload": "paper-table", "grid": f"icosahedral level {args.ico_level}",
                       "N": N, "err_samples": len(tg), "precision": "fp64"},
            "E_DS_EX": {nm: float(x) for nm, x in zip(names, e_ds)},
            "rows": rows,
            "ratio_ours_over_paper": {"median": float(np.median(ratios)),
                                      "min": float(ratios.min()), "max": float(ratios.max())}}


def run_runtime_table(args):
    """The paper's Table "runtimes" setting on the GPU: the N-body sum with
    the Laplace, biharmonic, Biot-Savart and SAL kernels (and the SAL kernel's
    leading term, the Newtonian kernel) on the icosahedral grid (level args.ico_level),
    CSFMM with MAC 0.7, degree 6, N0 = 144, in both precision forms (CUDA
    events, plan resident, median of 5), and the direct sum (FP32: all N^2
    pairs; FP64: sampled targets, scaled to N).  Prints the paper's serial CPU
    times beside them (context only: other hardware)."""
    import torch
    from paper_2508_13550_gb300 import csfmm as Cs
    from paper_2508_13550_gb300 import inputs as I
    pts, A = I.icosahedral_grid(args.ico_level)
    N = len(pts)
    dp = torch.from_numpy(pts).cuda()
    rng = np.random.default_rng(20250813)
    tg = torch.from_numpy(np.sort(rng.choice(N, min(args.err_samples, N), replace=False))
                          .astype(np.int64)).cuda()
    paper = {}
    with open(os.path.join(ROOT, "tests", "golden", "runtimes_table.txt")) as f:
        hdr = None
        for line in f:
            if line.startswith("# kernel"):
                hdr = [int(x.split("=")[-1]) for x in line.split()[3:]]
            line = line.split("#", 1)[0].split()
            if line:
                paper[(line[0], line[1])] = dict(zip(hdr, map(float, line[2:])))

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), out

    rows = []
    for name, paper_name, kid in (("Laplace", "Laplace", Cs.KERNEL_LAPLACE),
                                  ("biharmonic", "biharmonic", Cs.KERNEL_BIHARMONIC),
                                  ("Biot-Savart", "Biot-Savart", Cs.KERNEL_BIOT_SAVART),
                                  ("SAL", "SAL", Cs.KERNEL_SAL),
                                  ("Newtonian", "SAL", Cs.KERNEL_NEWTON)):
        f = I.rossby_haurwitz_vorticity(pts) if kid == Cs.KERNEL_BIOT_SAVART else \
            I.real_sph_harm(4, 3, pts)
        dw = torch.from_numpy(np.ascontiguousarray((f * A)[None])).cuda()
        ms_ds64, ds = timed(lambda: Cs.direct(dp, kid, dw, precision=Cs.FP64, targets=tg), 1)
        ms_ds32, _ = timed(lambda: Cs.direct(dp, kid, dw, precision=Cs.FP32_BULK), 1)
        row = {"kernel": name, "N": N, "direct_fp64_ms_scaled": ms_ds64 * N / len(tg),
               "direct_fp32_ms": ms_ds32,
               "paper_direct_s": paper[(paper_name, "direct")].get(N),
               "paper_csfmm_s": paper[(paper_name, "csfmm")].get(N)}
        for tag, prec in (("fp64", Cs.FP64), ("fp32", Cs.FP32_BULK)):
            P = Cs.plan_create(dp, kid, 6, 0.7, 144, precision=prec)
            ms, out = timed(lambda: Cs.evaluate(P, dw), 5)
            Cs.plan_destroy(P)
            row[f"csfmm_{tag}_ms"] = ms
            row[f"csfmm_{tag}_rel_err"] = float(torch.linalg.norm(out[:, tg] - ds)
                                                / torch.linalg.norm(ds))
        rows.append(row)
        log(row)
    return {"metric": "N-body sum runtime per kernel (Table runtimes setting)", "unit": "ms",
            "config": {"workload": "runtime-table", "grid": f"icosahedral level {args.ico_level}",
                       "N": N, "degree": 6, "theta": 0.7, "max_leaf": 144},
            "rows": rows,
            "paper_context": "serial CPU (one AMD EPYC 7763 core), FP64 C++"}


def run_bve(args):
    """The paper's BVE runs (Sec. 12) on the GPU: the RH wave-4 on the
    icosahedral grid of level args.bve_level (N = 163842 at level 7), RK4 with
    dt = 0.01 day and Omega = 2 pi per day, the velocity by the CSFMM (MAC 0.7,
    degree 6, N0 = 144; a plan built at every stage, the grid's plan reused
    for the first stage of remeshed steps) in both precision forms or by the
    direct sum, with and without remeshing onto the grid after every step.
    Times one RK4 step with CUDA events (median over args.steps steps after
    args.warmup; the FP64 direct step once) and reports E_zeta (Eq. bveerr)
    after args.bve_days days; then E_zeta of the remeshed method against N
    (levels 4 .. args.bve_level) with the CSFMM and the direct sum, the
    setting of the paper's Figure bveerr.  The paper's ratio (CSFMM 36x faster
    than the direct sum at N = 163842, serial CPU) is printed as context."""
    import torch
    from paper_2508_13550_gb300 import csfmm as Cs
    from paper_2508_13550_gb300 import inputs as I
    dt, om = I.BVE_DT, I.BVE_OMEGA
    nsteps = int(round(args.bve_days / dt))
    forms = {"csfmm_fp64": (6, Cs.FP64), "csfmm_fp32": (6, Cs.FP32_BULK),
             "direct_fp32": (0, Cs.FP32_BULK), "direct_fp64": (0, Cs.FP64)}

    def setup(level):
        x, z, A, off, nb = I.workload_bve(level, with_adjacency=True)
        dx, dz, dA = (torch.from_numpy(a).cuda() for a in (x, z, A))
        G = Cs.remesh_grid_create(dx, torch.from_numpy(off).cuda(), torch.from_numpy(nb).cuda())
        return x, z, A, dx, dz, dA, G

    def e_zeta(zs, xs, A):
        ex = I.rossby_haurwitz_vorticity(xs)
        return float(np.sqrt(np.sum((zs - ex) ** 2 * A) / np.sum(ex ** 2 * A)))

    def stepper(deg, prec, dx, dA, G, remeshed):
        plan = (Cs.plan_create(dx, Cs.KERNEL_BIOT_SAVART, deg, 0.7, 144, precision=prec,
                               max_nrhs=1) if remeshed and deg > 0 else None)
        if remeshed:
            return lambda xi, zi: (xi, Cs.bve_step_remeshed(G, zi, dA, dt, om, deg, 0.7, 144,
                                                            prec, grid_plan=plan))
        return lambda xi, zi: Cs.bve_step(xi, zi, dA, dt, om, deg, 0.7, 144, prec)

    def timed(step, dx, dz, k, w):
        xi, zi = dx, dz
        for _ in range(w):
            xi, zi = step(xi, zi)
        torch.cuda.synchronize()
        ts = []
        for _ in range(k):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            xi, zi = step(xi, zi)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    x, z, A, dx, dz, dA, G = setup(args.bve_level)
    N = len(x)
    if args.bve_quick:
        # remeshed CSFMM FP32-bulk steps only (the case the profiles break down)
        st = stepper(*forms["csfmm_fp32"], dx, dA, G, True)
        ms = timed(st, dx, dz, args.steps, args.warmup)
        return {"metric": "BVE remeshed RK4 step time, CSFMM FP32 bulk", "unit": "ms",
                "value": ms, "higher_is_better": False,
                "config": {"workload": "bve-rh-wave", "grid": f"icosahedral level {args.bve_level}",
                           "N": N, "dt_day": dt, "degree": 6, "theta": 0.7, "max_leaf": 144}}
    rows = {}
    for tag, (deg, prec) in forms.items():
        slow = tag == "direct_fp64"
        rows[tag] = {}
        for rm in (False, True):
            st = stepper(deg, prec, dx, dA, G, rm)
            ms = timed(st, dx, dz, 1 if slow else args.steps, 0 if slow else args.warmup)
            rows[tag]["ms_per_step_remeshed" if rm else "ms_per_step"] = ms
            log(tag, "remeshed" if rm else "", f"{ms:.2f} ms per RK4 step")
            if slow:
                continue
            xi, zi = dx, dz
            for _ in range(nsteps):
                xi, zi = st(xi, zi)
            torch.cuda.synchronize()
            e = e_zeta(zi.cpu().numpy(), xi.cpu().numpy(), A)
            rows[tag]["E_zeta_remeshed" if rm else "E_zeta"] = e
            log(tag, "remeshed" if rm else "", "E_zeta", e)
    conv = []
    for level in range(4, args.bve_level + 1):
        xl, zl, Al, dxl, dzl, dAl, Gl = (x, z, A, dx, dz, dA, G) if level == args.bve_level \
            else setup(level)
        row = {"level": level, "N": len(xl)}
        for tag in ("csfmm_fp32", "direct_fp32"):
            st = stepper(*forms[tag], dxl, dAl, Gl, True)
            zi = dzl
            for _ in range(nsteps):
                _, zi = st(dxl, zi)
            torch.cuda.synchronize()
            row[tag] = e_zeta(zi.cpu().numpy(), xl, Al)
        conv.append(row)
        log("E_zeta remeshed", row)
    # Table tracer_errors: tracer q = z, remeshed, FP64 CSFMM, Day 2
    paper_tr = {}
    with open(os.path.join(ROOT, "tests", "golden", "tracer_errors_table.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].split()
            if line:
                paper_tr[line[0]] = [float(v) for v in line[1:]]
    tracer = []
    for i, level in enumerate(range(5, args.bve_level + 1)):
        xl, zl, Al, dxl, dzl, dAl, Gl = (x, z, A, dx, dz, dA, G) if level == args.bve_level \
            else setup(level)
        plan = Cs.plan_create(dxl, Cs.KERNEL_BIOT_SAVART, 6, 0.7, 144, precision=Cs.FP64,
                              max_nrhs=1)
        zi, qi = dzl, dxl[:, 2].contiguous()
        for _ in range(2 * nsteps):
            zi, qi = Cs.bve_step_remeshed(Gl, zi, dAl, dt, om, 6, 0.7, 144, Cs.FP64,
                                          grid_plan=plan, tracer=qi)
        q = qi.cpu().numpy()
        row = {"level": level, "N": len(xl), "abs_mass": abs(float(np.sum(q * Al))),
               "qmax_minus_1": float(np.abs(q).max() - 1.0)}
        if i < 3:
            row["paper_abs_mass"] = paper_tr["abs_mass"][i]
            row["paper_qmax_minus_1"] = paper_tr["qmax_minus_1"][i]
        tracer.append(row)
        log("tracer Day 2", row)
    # Gaussian vortex (Eq. Gaussian_ic, Figure gv): remeshed CSFMM FP32 run, the
    # core's position (centroid of the vorticity above half its maximum) per day
    xg, zg, Ag, offg, nbg = I.workload_bve(args.bve_level, "gaussian", with_adjacency=True)
    dxg, dAg = torch.from_numpy(xg).cuda(), torch.from_numpy(Ag).cuda()
    Gg = Cs.remesh_grid_create(dxg, torch.from_numpy(offg).cuda(), torch.from_numpy(nbg).cuda())
    Pg = Cs.plan_create(dxg, Cs.KERNEL_BIOT_SAVART, 6, 0.7, 144, precision=Cs.FP32_BULK,
                        max_nrhs=1)

    def core(zv):
        wv = np.maximum(zv - 0.5 * zv.max(), 0.0) * Ag
        cv = (wv[:, None] * xg).sum(0)
        cv /= np.linalg.norm(cv)
        return [math.degrees(math.asin(cv[2])), math.degrees(math.atan2(cv[1], cv[0]))]

    track = [core(zg)]
    zi = torch.from_numpy(zg).cuda()
    for day in range(3):
        for _ in range(int(round(1.0 / dt))):
            zi = Cs.bve_step_remeshed(Gg, zi, dAg, dt, om, 6, 0.7, 144, Cs.FP32_BULK,
                                      grid_plan=Pg)
        torch.cuda.synchronize()
        track.append(core(zi.cpu().numpy()))
    log("Gaussian vortex core (lat, lon) by day", track)
    d64 = rows["direct_fp64"]["ms_per_step"]
    return {"metric": "BVE vortex-method RK4 step time (Sec. 12 setting)", "unit": "ms",
            "config": {"workload": "bve-rh-wave", "grid": f"icosahedral level {args.bve_level}",
                       "N": N, "dt_day": dt, "omega": om, "degree": 6, "theta": 0.7,
                       "max_leaf": 144, "days": args.bve_days, "remesh_ring": 2},
            "rows": rows,
            "speedup_over_direct_fp64": {k: d64 / v["ms_per_step"] for k, v in rows.items()},
            "E_zeta_remeshed_vs_N": conv,
            "tracer_day2": tracer,
            "gaussian_vortex_core_lat_lon_by_day": track,
            "paper_context": "CSFMM 36x faster than direct summation at N = 163842 "
                             "(serial CPU, FP64)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="newton-6m",
                    choices=sorted(WORKLOADS) + ["serving", "accuracy-sweep", "cstc-vs-fmm",
                                                 "paper-table", "runtime-table", "bve"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--err-samples", type=int, default=2048)
    ap.add_argument("--cpu-leaves", type=int, default=16384)
    ap.add_argument("--ref-leaves", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=5,
                    help="timed evaluations of the FP64 form on the same workload")
    ap.add_argument("--side-steps", type=int, default=10)
    ap.add_argument("--no-side-workloads", dest="side_workloads", action="store_false",
                    help="skip the Biot-Savart 393k and 16-RHS 1.5M workloads")
    ap.add_argument("--no-persistent", action="store_true",
                    help="several right-hand sides: per-phase launches instead of the "
                         "persistent launch")
    ap.add_argument("--no-fp64-compare", dest="fp64_compare", action="store_false")
    ap.add_argument("--schedule", type=int, default=0,
                    help="csfmm_options.schedule bits of the benchmarked plan (CSFMM_SCHED_*)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="multi-RHS workloads: keep the default leaf size and RHS chunk")
    ap.add_argument("--sweep-m", type=int, default=1024)
    ap.add_argument("--sweep-degrees", default="6,8,10,12")
    ap.add_argument("--ico-level", type=int, default=8)
    ap.add_argument("--bve-level", type=int, default=7)
    ap.add_argument("--bve-days", type=float, default=1.0)
    ap.add_argument("--bve-quick", action="store_true",
                    help="bve workload: time remeshed CSFMM FP32 steps only")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-sample", type=int, default=2000,
                    help="requests of the serving stream measured in the default line (0: none)")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-policy", default="cheapest", choices=["cheapest", "fifo"])
    ap.add_argument("--serve-age-ms", type=float, default=250.0)
    ap.add_argument("--serve-budget-gb", type=float, default=96.0)
    args = ap.parse_args()
    if args.warmup < 3:
        log("warning: fewer than 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "accuracy-sweep":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(run_accuracy_sweep(args)), flush=True)
        return 0
    if args.workload == "runtime-table":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(run_runtime_table(args)), flush=True)
        return 0
    if args.workload == "bve":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(run_bve(args)), flush=True)
        return 0
    if args.workload == "paper-table":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(run_paper_table(args)), flush=True)
        return 0
    if args.workload == "cstc-vs-fmm":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(run_cstc_vs_fmm(args)), flush=True)
        return 0
    if args.workload == "serving":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        summ = run_serving(args)
        print(json.dumps({"metric": "serving p50/p99 latency", "value": summ["p99_ms"],
                          "unit": "ms (p99)", "higher_is_better": False, "n_gpus": 1,
                          "dtype": "f32", "data": "synthetic",
                          "config": {"workload": "serving", "requests": summ["requests"]},
                          "serving": summ}), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
