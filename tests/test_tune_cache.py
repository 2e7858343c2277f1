"""The autotuner's cache file, read on the host (csfmm_tune_cache_read; no
GPU work): valid lines are found (the last one for a key wins), and lines of
a stale format, with values out of range, cut short or carrying trailing
text are ignored instead of misconfiguring a plan."""
import pytest

from paper_2508_13550_gb300 import csfmm as C

KEY = "NVIDIA_GB300|k0|n10|t0.7|p1|r16|N1572864"
GOOD = f"v2 {KEY} 400 16 0 0 20.5 5.1e-08 20.6 5.1e-08\n"


@pytest.fixture(scope="module")
def lib():
    try:
        return C.load()
    except RuntimeError as e:
        pytest.skip(str(e))


def _write(tmp_path, text):
    p = tmp_path / "tune.txt"
    p.write_text(text)
    return str(p)


def test_valid_line_is_read(lib, tmp_path):
    r = C.tune_cache_read(_write(tmp_path, GOOD), KEY)
    assert r["max_leaf"] == 400 and r["rhs_chunk"] == 16 and r["no_persistent"] == 0
    assert r["schedule"] == 0 and r["from_cache"] == 1 and r["ms_per_eval"] == 20.5
    # the last valid line for the key wins; other keys are not confused with it
    text = GOOD + f"v2 {KEY}x 100 8 1 5 1 1 1 1\n" + f"v2 {KEY} 256 8 1 6 19.0 5e-08 20.6 5.1e-08\n"
    r = C.tune_cache_read(_write(tmp_path, text), KEY)
    assert (r["max_leaf"], r["rhs_chunk"], r["no_persistent"], r["schedule"]) == (256, 8, 1, 6)


@pytest.mark.parametrize("bad", [
    f"{KEY} 400 16 20.5 5.1e-08 20.6 5.1e-08\n",              # stale format of an earlier version
    f"v1 {KEY} 400 16 0 0 20.5 5.1e-08 20.6 5.1e-08\n",       # unknown version tag
    f"v2 {KEY} 400 16 0 0 20.5\n",                            # cut short
    f"v2 {KEY} 0 16 0 0 20.5 5.1e-08 20.6 5.1e-08\n",         # leaf size out of range
    f"v2 {KEY} 400 12 0 0 20.5 5.1e-08 20.6 5.1e-08\n",       # chunk not 0/4/8/16
    f"v2 {KEY} 400 16 2 0 20.5 5.1e-08 20.6 5.1e-08\n",       # flag not 0/1
    f"v2 {KEY} 400 16 0 128 20.5 5.1e-08 20.6 5.1e-08\n",     # schedule bits out of range
    f"v2 {KEY} 400 16 0 0 nan 5.1e-08 20.6 5.1e-08\n",        # not finite
    f"v2 {KEY} 400 16 0 0 -1 5.1e-08 20.6 5.1e-08\n",         # negative time
    f"v2 {KEY} 400 16 0 0 20.5 5.1e-08 20.6 5.1e-08 junk\n",  # trailing text
    "\x00\xff garbage " * 200 + "\n",                          # binary junk, longer than a line
    f"v2 {KEY} 400 16 0 0 20.5\x00 5.1e-08 20.6 5.1e-08\n",   # a NUL byte inside
])
def test_corrupt_or_stale_lines_are_ignored(lib, tmp_path, bad):
    assert C.tune_cache_read(_write(tmp_path, bad), KEY) is None
    # a corrupt line does not hide a valid one before or after it
    assert C.tune_cache_read(_write(tmp_path, GOOD + bad), KEY)["max_leaf"] == 400
    assert C.tune_cache_read(_write(tmp_path, bad + GOOD), KEY)["max_leaf"] == 400


def test_missing_file_and_arguments(lib, tmp_path):
    assert C.tune_cache_read(str(tmp_path / "none.txt"), KEY) is None
    res = C.TuneResult()
    assert lib.csfmm_tune_cache_read(None, KEY.encode(), res) == 1
