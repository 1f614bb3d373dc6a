"""Host logic of the benchmark's roofline object (no GPU): the fraction is
the algorithmic bytes of the method (16 FP64 field passes of 25 fields per
RK4 step, 800 B per zone and stage on average) over the stage kernel's
launch time, against the measured HBM peak, in both precisions; FP64 adds
its FP64-pipe use; the traffic comes from the ncu captures of the stage
kernels the levels use and is null when a level uses a kernel without one."""
import bench


def _run(precision, ids):
    kern = {"name": "k", "ms": 0.5, "launches": 508, "steps": 1, "zones_per_launch": 884736.0,
            "bytes_per_launch": 884736.0 * 800, "flops_per_launch": 884736.0 * 5355 if precision == "fp64" else None,
            "kernel_ids_used": ids, "stage_kernels": ["x"] * 7}
    return {"precision": precision, "kern": kern, "ms": 280.0}


def test_traffic_from_captured_kernels(monkeypatch):
    monkeypatch.setattr(bench, "NCU_TRAFFIC_PER_ZONE", {(1, 10): 1000.0, (1, 11): 1100.0, (0, 0): 2000.0})
    r = bench.roofline(_run("mixed", [10]), 6657.6)
    assert r["bound"] == "hbm" and abs(r["traffic"] - 1000.0 * 884736) < 1.0
    r = bench.roofline(_run("mixed", [10, 11]), 6657.6)  # the larger of the two captures
    assert abs(r["traffic"] - 1100.0 * 884736) < 1.0
    r = bench.roofline(_run("fp64", [0]), 6657.6)
    assert r["bound"] == "hbm" and r["limited_by"] == "FP64 pipe" and abs(r["traffic"] - 2000.0 * 884736) < 1.0


def test_no_traffic_for_uncaptured_kernel(monkeypatch):
    monkeypatch.setattr(bench, "NCU_TRAFFIC_PER_ZONE", {(1, 10): 1000.0})
    assert bench.roofline(_run("mixed", [10, 12]), 6657.6)["traffic"] is None
    assert bench.roofline(_run("mixed", []), 6657.6)["traffic"] is None


def test_fraction_is_algorithmic_bytes_over_peak():
    """3200 B per zone update (one RK4 step) = 800 B per zone per stage, the
    same for both precisions; the mixed path's own hi/lo copies are reported
    beside it, not in the fraction."""
    assert bench.BYTES_PER_ZONE_UPDATE == 3200 and bench.ALG_BYTES_PER_ZONE_STAGE == 800
    for prec in ("mixed", "fp64"):
        r = bench.roofline(_run(prec, [10 if prec == "mixed" else 0]), 6657.6)
        assert abs(r["achieved"] - 884736.0 * 800 / 0.5e-3 / 1e9) < 1e-6
        assert abs(r["frac"] - r["achieved"] / 6657.6) < 1e-12
    r = bench.roofline(_run("fp64", [0]), 6657.6)
    assert abs(r["alu"]["achieved"] - 884736.0 * 5355 / 0.5e-3 / 1e12) < 1e-9
    assert abs(r["alu"]["frac"] - r["alu"]["achieved"] / 1.25) < 1e-12


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
