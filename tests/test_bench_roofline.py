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


def test_launches_per_coarse_step_by_recursion():
    """The launch count the bench reports for one coarse step, counted by
    walking the Berger-Oliger recursion: per level step 4 stage kernels, the
    ghost work (4 Sommerfeld updates on level 0; on finer levels fills for
    stage 1, stages 2-3 together and stage 4), the level bookkeeping and,
    with children, the prolongation of the new slot; per child level step
    pair the fill at the new time, the restriction and the prolongation of
    the restricted slot.  1269 launches for the 7-level binary (the ncu
    launch list of the step has exactly these)."""
    import initial_data as idd
    h = idd.binary_7_level()
    nlev = len(h.levels)

    def level_step(l):
        n = 4 + (4 if l == 0 else 3) + 1
        if l + 1 < nlev:
            n += 1 + level_step(l + 1) + level_step(l + 1) + 3
        return n

    assert level_step(0) == bench.launches_per_coarse_step(h) == 1269
