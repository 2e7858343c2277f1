"""The bounds-checked build (-DCSFMM_CHECKED), the stand-in for a memory
checker: every cell index a kernel takes from an interaction list, a leaf
table or a child slot is validated, and a bad one would set the plan's status
word (CSFMM_ERR_DEVICE) instead of being read.  Every evaluation path runs
here with the checked library in a child process: no check fires and the
results equal the unchecked library's bit for bit (the checks change no
arithmetic)."""
import os
import subprocess
import sys

import pytest

from gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2508_13550_gb300 import csfmm as C, inputs as I
C.load(sys.argv[2])
out = {}
pts, A = I.cubed_sphere_grid(40)
rnd = I.random_sphere_points(9000, 3)
for name, p, kid, prec, nrhs, extra in [
        ("fp64", pts, 0, C.FP64, 2, {}), ("fp32-sym", pts, 2, C.FP32_BULK, 1, {}),
        ("fp32-bs", rnd, 1, C.FP32_BULK, 3, {}), ("fp32-persistent", pts, 0, C.FP32_BULK, 16, {}),
        ("fp32-per-phase", rnd, 2, C.FP32_BULK, 8, {"no_persistent": True}),
        ("fp32-shrunk", rnd, 3, C.FP32_BULK, 1, {"shrink": True})]:
    W = np.random.default_rng(5).standard_normal((nrhs, len(p))) / len(p)
    P = C.plan_create(torch.from_numpy(p).cuda(), kid, 7, 0.7, 60, precision=prec, max_nrhs=nrhs,
                      **extra)
    dW = torch.from_numpy(W).cuda()
    out[name] = C.evaluate(P, dW).cpu().numpy()
    out[name + "-cstc"] = C.evaluate_cstc(P, dW).cpu().numpy()
    C.plan_sync(P)  # raises CSFMM_ERR_DEVICE if a check fired
np.savez(sys.argv[3], **out)
"""


def test_checked_build_runs_clean_and_bitwise(tmp_path):
    cuda_or_skip()
    from paper_2508_13550_gb300 import build as B
    checked = B.build(checked=True)
    res = {}
    for tag, lib in (("checked", checked), ("plain", B.LIB)):
        f = str(tmp_path / f"{tag}.npz")
        r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, lib, f], capture_output=True,
                           text=True, timeout=900)
        assert r.returncode == 0, r.stderr[-3000:]
        import numpy as np
        res[tag] = dict(np.load(f))
    for k in res["plain"]:
        assert (res["checked"][k] == res["plain"][k]).all(), k
