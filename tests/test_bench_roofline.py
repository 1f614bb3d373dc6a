"""Host logic of the benchmark's roofline object (no GPU): the traffic of
the dominant kernel comes from the ncu captures of the stage kernels the
levels use, and is null when a level uses a kernel without a capture."""
import bench


def _run(precision, ids):
    kern = {"name": "k", "ms": 0.5, "launches": 508, "steps": 1, "zones_per_launch": 884736.0,
            "bytes_per_launch": 884736.0 * 900, "flops_per_launch": 884736.0 * 5355 if precision == "fp64" else None,
            "kernel_ids_used": ids, "stage_kernels": ["x"] * 7}
    return {"precision": precision, "kern": kern, "ms": 280.0}


def test_traffic_from_captured_kernels():
    r = bench.roofline(_run("mixed", [10]), 6657.6)
    assert r["bound"] == "hbm" and abs(r["traffic"] - 0.8531e9) < 1.0
    r = bench.roofline(_run("mixed", [10, 11]), 6657.6)  # the larger of the two captures
    assert abs(r["traffic"] - 0.8531e9) < 1.0
    r = bench.roofline(_run("fp64", [0]), 6657.6)
    assert r["bound"] == "alu" and abs(r["traffic"] - 1.98e9) < 1.0


def test_no_traffic_for_uncaptured_kernel():
    assert bench.roofline(_run("mixed", [10, 12]), 6657.6)["traffic"] is None
    assert bench.roofline(_run("mixed", []), 6657.6)["traffic"] is None


def test_fraction_is_achieved_over_peak():
    r = bench.roofline(_run("mixed", [10]), 6657.6)
    assert abs(r["achieved"] - 884736.0 * 900 / 0.5e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6657.6) < 1e-12
