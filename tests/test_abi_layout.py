"""The Python binding's ctypes structures have the C header's layout: a small
C program compiled against include/csfmm.h prints sizeof and offsetof of every
field, and the ctypes classes must agree (no GPU, no CUDA library needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

PAIRS = [("Options", "csfmm_options"), ("Stats", "csfmm_stats"),
         ("TuneResult", "csfmm_tune_result"), ("Request", "csfmm_request"),
         ("RequestTiming", "csfmm_request_timing"), ("ServerStats", "csfmm_server_stats")]


def test_ctypes_structures_match_the_header(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no host C compiler")
    from paper_2508_13550_gb300 import csfmm
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "csfmm.h"',
             "int main(void) {"]
    for py, c in PAIRS:
        cls = getattr(csfmm, py)
        lines.append(f'  printf("{c} %zu\\n", sizeof({c}));')
        for name, _ in cls._fields_:
            lines.append(f'  printf("{c}.{name} %zu\\n", offsetof({c}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", str(exe), str(src)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for py, c in PAIRS:
        cls = getattr(csfmm, py)
        assert int(got[c]) == ctypes.sizeof(cls), c
        for name, _ in cls._fields_:
            assert int(got[f"{c}.{name}"]) == getattr(cls, name).offset, f"{c}.{name}"
