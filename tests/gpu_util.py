"""Helpers of the GPU tests: skip without a GPU, host/device conversion."""
import numpy as np
import pytest


def cuda_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_13550_gb300 import csfmm
    csfmm.load()
    return torch


def dev(torch, a, dtype=None):
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a)
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def cell_keys(C):
    return [(int(f), int(l), int(a), int(b)) for f, l, a, b in
            zip(C["face"], C["level"], C["ia"], C["ib"])]
