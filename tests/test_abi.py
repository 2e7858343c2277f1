"""CPU-side checks of the boundary: the CUDA library builds for sm_103a,
loads, and exports every entry point that include/csfmm.h declares.  No
compute call is made (there may be no GPU)."""
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "csfmm.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(csfmm_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2508_13550_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("csfmm_plan_create", "csfmm_evaluate", "csfmm_direct",
                     "csfmm_plan_destroy", "csfmm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(csfmm_[a-z_0-9]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2508_13550_gb300 import csfmm
    lib = csfmm.load(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)
        assert n in csfmm.exported_symbols()
    assert "sm_103a" in csfmm.version()


def test_library_is_built_for_sm103a_only(lib_path):
    from paper_2508_13550_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
