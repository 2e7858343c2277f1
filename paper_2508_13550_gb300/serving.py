"""Drives the library's serving loop (csfmm_server_*) with a seeded request
stream and reports latency percentiles and throughput.

Inputs live on the device: for every grid size m the cubed-sphere points, the
cell areas and a few smooth basis fields (random real spherical-harmonic
combinations from inputs.py).  A request's weights are a seeded linear
combination of the basis fields times the cell areas, built on the device
just before it is submitted.  Requests are submitted at their arrival times
(a Poisson process); the library admits them as slots and memory free up and
runs admitted requests concurrently.  Latency = completion - submission on
the library's host clock.
"""
from __future__ import annotations

import time

import numpy as np

from . import csfmm as C
from . import inputs as I


class DeviceGrids:
    """Per grid size m: points [N,3], areas [N] and K basis fields [K,N] on
    the device."""

    def __init__(self, ms, device, nbasis: int = 4, nmax: int = 4, seed: int = I.MASTER_SEED):
        import torch
        self.device = device
        self.grids = {}
        for m in ms:
            pts, A = I.cubed_sphere_grid(int(m))
            coeffs = I.random_sh_coeffs(nmax, nbasis, seed + int(m))
            B = I.sph_harm_combination(pts, coeffs, nrhs=nbasis)
            self.grids[int(m)] = (torch.from_numpy(pts).to(device),
                                  torch.from_numpy(A).to(device),
                                  torch.from_numpy(np.ascontiguousarray(B)).to(device))

    def points(self, m):
        return self.grids[m][0]

    def weights(self, m, nrhs, seed):
        import torch
        pts, A, B = self.grids[m]
        g = torch.Generator(device="cpu").manual_seed(int(seed))
        c = torch.randn((nrhs, B.shape[0]), generator=g, dtype=torch.float64).to(self.device)
        return ((c @ B) * A[None, :]).contiguous()


def leaf_size(degree: int) -> int:
    """The paper's default maximum leaf size N0 = 4 n^2 (Sec. 10)."""
    return 4 * degree * degree


def run_stream(server: C.Server, grids: DeviceGrids, requests, rate_hz=None, theta=0.7,
               precision=C.FP32_BULK, max_outstanding=64, keep_outputs=False, stream=None):
    """Submits `requests` (dicts from inputs.serving_requests) at their arrival
    times scaled to rate_hz (None: all at once) and waits for all.  Returns a
    list of per-request records (and outputs if keep_outputs)."""
    import torch
    if not requests:
        return []
    base_rate = len(requests) / max(requests[-1]["arrival"], 1e-9)
    scale = 0.0 if rate_hz is None else base_rate / rate_hz
    t0 = time.perf_counter()
    outstanding = {}
    records = []

    def reap(block_oldest=False):
        done_ids = []
        for rid, (req, w, out) in outstanding.items():
            done, t = server.poll(rid)
            if done:
                done_ids.append((rid, t))
        if not done_ids and block_oldest:
            rid = next(iter(outstanding))
            rc, t = server.wait(rid)
            done_ids.append((rid, t))
        for rid, t in done_ids:
            req, w, out = outstanding.pop(rid)
            rec = dict(req)
            rec.update(t)
            rec["latency_ms"] = t["done_ms"] - t["submit_ms"]
            if keep_outputs:
                rec["out"] = out.cpu().numpy()
                rec["weights"] = w.cpu().numpy()
            records.append(rec)

    for req in requests:
        target = t0 + req["arrival"] * scale
        while True:
            now = time.perf_counter()
            if now >= target:
                break
            if outstanding:
                reap()
            time.sleep(min(2e-4, max(0.0, target - now)))
        while len(outstanding) >= max_outstanding:
            reap(block_oldest=True)
        m, kid, nrhs, deg = req["m"], req["kernel"], req["nrhs"], req["degree"]
        w = grids.weights(m, nrhs, req["seed"])
        out = torch.empty((nrhs, w.shape[1], C.kernel_dim(kid)), dtype=torch.float64,
                          device=w.device)
        torch.cuda.current_stream().synchronize()  # weights ready before the server reads them
        rid = server.submit(grids.points(m), m, kid, deg, theta, leaf_size(deg), precision, w, out)
        outstanding[rid] = (req, w, out)
    while outstanding:
        reap(block_oldest=True)
    return records


def summarize(records):
    """p50/p99 latency (ms), aggregate targets/s (sum of N * nrhs over the
    span from first submission to last completion) and request rate, and the
    latency percentiles and median GPU time per grid size m."""
    lat = np.array([r["latency_ms"] for r in records])
    ms = np.array([r["m"] for r in records])
    gpu = np.array([r["gpu_ms"] for r in records])
    first = min(r["submit_ms"] for r in records)
    last = max(r["done_ms"] for r in records)
    span_s = (last - first) / 1e3
    targets = sum(6 * r["m"] ** 2 * r["nrhs"] for r in records)
    return {
        "requests": len(records),
        "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()),
        "max_ms": float(lat.max()),
        "span_s": span_s,
        "targets_per_s": targets / span_s,
        "requests_per_s": len(records) / span_s,
        "failed": int(sum(1 for r in records if r["status"] != 0)),
        "plans_built_in_stream": int(sum(r["built_plan"] for r in records)),
        "by_grid_size": {
            int(m): {"requests": int((ms == m).sum()),
                     "p50_ms": float(np.percentile(lat[ms == m], 50)),
                     "p99_ms": float(np.percentile(lat[ms == m], 99)),
                     "gpu_ms_p50": float(np.percentile(gpu[ms == m], 50))}
            for m in sorted(set(ms.tolist()))},
    }
