"""The bench's DRAM traffic table (ncu bytes per kernel evaluation) belongs to
the interaction kernels' current sources: the hash it records must match them,
so that a kernel edited since the capture reports no traffic rather than a
stale figure, and the committed table is the one captured from the committed
kernels."""
import bench


def test_traffic_table_matches_the_kernel_sources():
    for k in ("pp_sym_kernel", "near32x2_kernel", "far32x2_kernel", "cc_sym_kernel"):
        t = bench.traffic_per_launch(k, 1e9)
        assert t is not None and 0.0 < t < 1e9, k  # well under one byte per evaluation


def test_unknown_kernel_has_no_traffic():
    assert bench.traffic_per_launch("no_such_kernel", 1e9) is None
