"""Every ctypes signature of the Python binding matches its prototype in
include/csfmm.h: the same number of arguments, and each of the same kind
(pointer or handle, 32-bit integer, 64-bit integer, double).  A mismatch would
pass wrong bits through the C ABI without any error, so it is checked here on
the CPU."""
import ctypes
import os
import re

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "csfmm.h")
HANDLES = {"csfmm_plan", "csfmm_workspace", "csfmm_server", "csfmm_remesh_grid"}


def prototypes():
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\b(csfmm_[a-z_0-9]+)\s*\(([^()]*)\)\s*;", txt):
        args = [a.strip() for a in m.group(2).split(",")]
        out[m.group(1)] = [] if args == ["void"] or args == [""] else args
    return out


def c_kind(decl):
    decl = " ".join(decl.replace("*", " * ").split())
    words = decl.split()
    if "*" in words or words[0] in HANDLES or (len(words) > 1 and words[-2] in HANDLES):
        return "ptr"
    base = [w for w in words[:-1] if w != "const"]
    if base in (["double"],):
        return "f64"
    if base in (["int64_t"], ["uint64_t"]):
        return "i64"
    if base in (["int"], ["int32_t"], ["csfmm_status"]):
        return "i32"
    raise AssertionError(f"unclassified parameter {decl!r}")


def py_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or isinstance(t, type) and issubclass(
            t, ctypes._Pointer):
        return "ptr"
    if t is ctypes.c_double:
        return "f64"
    if t in (ctypes.c_int64, ctypes.c_uint64):
        return "i64"
    if t in (ctypes.c_int, ctypes.c_int32):
        return "i32"
    raise AssertionError(f"unclassified ctypes type {t!r}")


def test_binding_signatures_match_the_header():
    from paper_2508_13550_gb300 import csfmm
    protos = prototypes()
    assert len(protos) >= 20
    for name, argtypes in csfmm._SIGS.items():
        assert name in protos, name
        want = [c_kind(a) for a in protos[name]]
        got = [py_kind(t) for t in argtypes]
        assert got == want, f"{name}: binding {got} vs header {want}"
    assert set(protos) == set(csfmm._SIGS)
