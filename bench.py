"""Throughput benchmark of the Z4c hot path on GB300.

One step = one coarse step of the 7-level box-in-box Berger-Oliger hierarchy
around an equal-mass Brill-Lindquist binary (L0-L4: one 96^3 patch each,
dx = 4 .. 1/4; L5-L6: two 64^3 patches around the punctures at (+-5, 0, 0)):
127 level steps of RK4 with ghost prolongation, restriction and the
Sommerfeld outer boundary, recorded once as a CUDA graph and replayed.
77,758,464 zone updates per step (the paper's ZCPS count: sum over levels of
2^l x active cells).  value = zone updates / s over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Multi-GPU: replicas only (each rank evolves its own hierarchy; no collective
on the data path), launched by torchrun.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Z4c zone-updates/s per RK4 step, FP64 vs mixed; % of GB300 HBM roofline"
UNIT = "zone-updates/s"
WORKLOAD = "7-level box-in-box BO binary (BL m1=m2=0.5, sep 10M), one coarse step"
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 (profiling recipe); measured FMA probe: 1.0
# algorithmic HBM bytes per zone per RK stage (25 FP64 fields): stage 1 reads
# u_n and writes y and u_2 (3 passes), stages 2-3 read u_s, u_n, y and write
# y, u_s+1 (5), stage 4 reads u_4, y and writes u_n+1 (3): 16 passes per step
BYTES_PER_ZONE_UPDATE = 16 * 25 * 8
# mixed precision (FP32 hi/lo pairs, 8 B per value): stage 1 reads the split
# (hi_n, lo_n) and u_n (FP64), writes y (FP64) and the stage-2 pairs: 800 B;
# stages 2-3 read the stage pairs, (hi_n, lo_n) and y, write y and the next
# pairs: 1000 B; stage 4 reads the stage pairs and y, writes u_n+1 and its
# split: 800 B.  3600 B per zone update.
BYTES_PER_ZONE_UPDATE_MIXED = 3600


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                           "--format=csv,noheader,nounits", "-lms", "200"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self._proc = None
        return self

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(ms: float, dist) -> float:
    """The slowest rank's time (replicas: every rank times its own hierarchy;
    one all-reduce outside the timed region).  NCCL reduces a CUDA tensor,
    gloo a CPU one."""
    if not dist:
        return ms
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(zone_updates_per_rank: int, world: int, ms: float) -> float:
    """Zone updates of all ranks per second of the slowest rank."""
    return world * zone_updates_per_rank / (ms * 1e-3)


def hierarchy():
    import initial_data as idd
    return idd.binary_7_level()


def launches_per_coarse_step(h) -> int:
    """Kernels launched by one coarse step (the recursion is static): per level
    step 4 fused stage kernels, 3 ghost time fills on levels > 0 (stages 2 and
    3 share one), 4 Sommerfeld ghost updates on level 0, the level
    bookkeeping, the spatial prolongation of the new slot for the children;
    per child level step pair: ghost fill at the new time, restriction and the
    prolongation of the restricted slot.  (No same-level overlaps in these
    hierarchies, so no exchange launches.)"""
    total = 0
    nlev = len(h.levels)
    for l, lv in enumerate(h.levels):
        per = 4 + (3 if l > 0 else 4) + 1
        if l + 1 < nlev:
            per += 1 + 3  # prolong new slot; after the two child steps: fill, restrict, prolong
        total += (2 ** l) * per
    return total


def cpu_sample(steps: int = 1, n: int = 96, threads: int = 0):
    """The oracle (as it stands) on a bounded sample of the workload: RK4
    steps of the level-0 patch (96^3, or its central n^3) with its Sommerfeld
    ghosts, on all host cores or on `threads` of them."""
    import initial_data as idd
    import oracle
    h = hierarchy()
    p0 = h.levels[0][0]
    p = p0 if n == p0.n[0] else idd.centred_patch(n, p0.dx)
    u = idd.punctures(p, h.masses, h.positions)
    prm = oracle.Params()
    all_threads = oracle.num_threads()
    if threads:
        oracle.set_num_threads(threads)
    try:
        oracle.rk4_step(p, u, 0.25 * p.dx, prm)  # warm (builds the oracle)
        t0 = time.perf_counter()
        for _ in range(steps):
            u = oracle.rk4_step(p, u, 0.25 * p.dx, prm)
        dt = time.perf_counter() - t0
        used = oracle.num_threads()
    finally:
        if threads:
            oracle.set_num_threads(all_threads)
    zu = steps * p.active_points
    return zu / dt, used, "%d RK4 step(s) of the level-0 patch%s (%d zone updates)" % (
        steps, "" if n == p0.n[0] else ", its central %d^3" % n, zu)


def cpu_baseline(line_unit):
    """cpu_baseline of the bench line: the oracle on all host cores (one RK4
    step of the level-0 96^3 patch) and on one core (its central 48^3)."""
    v, cores, sample = cpu_sample(1)
    v1, _, sample1 = cpu_sample(1, n=48, threads=1)
    return {"value": v, "unit": line_unit, "cores": cores, "kind": "oracle", "sample": sample,
            "one_core": {"value": v1, "unit": line_unit, "cores": 1, "sample": sample1}}


def cpu_coarse_step_case(args):
    """The oracle's time for one full coarse step of the 7-level binary
    (BOHierarchy, all host cores, 77.76 M zone updates): long, not part of
    the default run."""
    import initial_data as idd
    import oracle
    h = hierarchy()
    states = idd.hierarchy_data(h)
    bo = oracle.BOHierarchy(h, states, oracle.Params(), courant=args.courant)
    t0 = time.perf_counter()
    bo.level_step(0)
    dt = time.perf_counter() - t0
    zu = h.zone_updates_per_coarse_step()
    print(json.dumps({"case": "cpu-coarse-step", "seconds": dt, "zone_updates": zu,
                      "zone_updates_per_s": zu / dt, "cores": oracle.num_threads()}), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_sample(1)
    vals = []
    cores = 1
    sample = ""
    for _ in range(args.steps):
        v, cores, sample = cpu_sample(1)
        vals.append(v)
    value = float(np.mean(vals))
    ms = 96 ** 3 / value * 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"],
                    help="both: value = mixed precision, with the FP64 run beside it")
    ap.add_argument("--courant", type=float, default=0.25)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--kernel", type=int, default=None,
                    help="force this stage kernel (ids of STAGE_KERNELS) on every level, no autotuning")
    ap.add_argument("--serial-ghosts", action="store_true",
                    help="refined levels' ghost fills and prolongation on the grid's stream, in order "
                         "(default: beside the stage kernels on a second stream)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default stage kernels instead of timing them first")
    ap.add_argument("--sizes", default="32,64,128", help="gauge-wave / robust-stability grid sizes")
    ap.add_argument("--sweep-sizes", default="48,64,96,128,160,192", help="sweep: single-patch sizes")
    ap.add_argument("--no-coarse", action="store_true", help="sweep: skip the full 10-level coarse step")
    ap.add_argument("--gw-steps", type=int, default=1000,
                    help="gauge-wave: RK4 steps on the coarsest grid; robust-stability: steps per grid")
    ap.add_argument("--case", default="amr7",
                    choices=["amr7", "uniform96", "mixed-error", "gauge-wave", "robust-stability", "sweep", "tov", "tov-amr",
                             "tov-moving",
                             "cpu-coarse-step",
                             "amr7-zsym", "adm", "amr7-moving", "psi4"],
                    help="uniform96: RK4 steps of one 96^3 puncture patch only (for ncu captures); "
                         "mixed-error: the 7-level hierarchy in FP64 and mixed precision side by side")
    ap.add_argument("--coarse-steps", type=int, default=64, help="mixed-error: coarse steps")
    ap.add_argument("--error-kernels", default="", help="mixed-error: stage kernels to compare, e.g. 6,0")
    ap.add_argument("--fp64-twin", action="store_true",
                    help="mixed-error: also an FP64 run from data perturbed at 1e-7 (FP32 rounding size)")
    ap.add_argument("--adm-steps", type=int, default=2, help="adm: coarse steps evolved before the integrals")
    ap.add_argument("--tov-n", type=int, default=128, help="tov: cells per axis of the patch on [-16, 16]^3")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.case == "cpu-coarse-step":
        if rank == 0:
            cpu_coarse_step_case(args)
        return

    import torch
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2607_08743_gb300 import build as skbuild
    skbuild.build()
    import paper_2607_08743_gb300 as sk

    if args.case == "uniform96":
        uniform_case(torch, sk, args)
        return
    if args.case == "mixed-error":
        mixed_error_case(torch, sk, args)
        return
    if args.case == "amr7-zsym":
        zsym_case(torch, sk, args)
        return
    if args.case == "sweep":
        sweep_case(torch, sk, args)
        return
    if args.case == "gauge-wave":
        gauge_wave_case(torch, sk, args)
        return
    if args.case == "robust-stability":
        robust_stability_case(torch, sk, args)
        return
    if args.case == "adm":
        adm_case(torch, sk, args)
        return
    if args.case == "amr7-moving":
        moving_case(torch, sk, args)
        return
    if args.case == "psi4":
        psi4_case(torch, sk, args)
        return
    if args.case == "tov-amr":
        return tov_amr_case(torch, sk, args)
    if args.case == "tov-moving":
        return tov_moving_case(torch, sk, args)
    if args.case == "tov":
        tov_case(torch, sk, args)
        return

    h = hierarchy()
    zu = h.zone_updates_per_coarse_step()
    precisions = ["mixed", "fp64"] if args.precision == "both" else [args.precision]
    runs = {}
    with ClockSampler(local) as clk:
        for p in precisions:
            runs[p] = measure(torch, sk, h, p, args, world, dist)
    head = runs[precisions[0]]
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if precisions[0] == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "levels": len(h.levels), "patches": len(h.patches),
                       "zone_updates_per_step": zu, "courant": args.courant, "precision": precisions[0],
                       "ghost_schedule": "serial" if args.serial_ghosts else "overlapped",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2: %.2f GB per state copy" % (
                           sum(25 * 8 * (p.n[0] + 6) * (p.n[1] + 6) * (p.n[2] + 6) for p in h.patches) / 1e9),
                       "hbm_roofline_zone_updates_per_s": hbm * 1e9 / BYTES_PER_ZONE_UPDATE,
                       "step_hbm_frac_of_measured": head["value"] / world / (hbm * 1e9 / BYTES_PER_ZONE_UPDATE)},
            "roofline": roofline(head, hbm),
            "gpu_launches": launches_per_coarse_step(h) * args.steps * len(precisions),
            "clocks": clk.summary(),
            "constraints_l0": head["constraints_l0"]}
    if head.get("e2e"):
        line["e2e"] = head["e2e"]
    for p in precisions[1:]:
        r = runs[p]
        line[p] = {"value": r["value"], "ms_per_step": r["ms"], "dtype": "f64" if p == "fp64" else "f32+f64",
                   "roofline": roofline(r, hbm), "constraints_l0": r["constraints_l0"]}
        if r.get("e2e"):
            line[p]["e2e"] = r["e2e"]
    if len(precisions) > 1:
        line["speedup_mixed_over_fp64"] = runs["mixed"]["value"] / runs["fp64"]["value"]
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(UNIT)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# per-zone DRAM traffic of the stage kernel (ncu dram__bytes_read + write of
# the four RK4 stage launches of one step on the 96^3 patch, averaged over
# the stages, divided by its 884,736 zones), by (precision, stage kernel id);
# the captures are in profiles/.  A kernel without a capture reports no
# traffic; levels on different captured kernels report the largest.
NCU_TRAFFIC_PER_ZONE = {(0, 0): 1183.6, (1, 10): 1064.6, (1, 20): 1103.5}
# the metric's roofline: the algorithmic bytes of one RK4 step (16 FP64
# field passes of 25 fields) per zone update, the same in both precisions
# (the hi/lo split copies of mixed precision are an implementation choice)
ALG_BYTES_PER_ZONE_STAGE = BYTES_PER_ZONE_UPDATE / 4.0


def roofline(r, hbm):
    """The dominant kernel (the fused RHS + RK4 stage) against the HBM
    roofline of the algorithmic bytes; FP64 adds its FP64-pipe use, the
    resource that limits it."""
    k = r["kern"]
    alg = k["zones_per_launch"] * ALG_BYTES_PER_ZONE_STAGE
    ach = alg / (k["ms"] * 1e-3) / 1e9
    out = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
           "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs)",
           "algorithmic_bytes_per_zone_stage": ALG_BYTES_PER_ZONE_STAGE}
    if r["precision"] == "fp64":
        fl = k["flops_per_launch"] / (k["ms"] * 1e-3) / 1e12 if k["flops_per_launch"] else None
        out["limited_by"] = "FP64 pipe"
        out["alu"] = {"achieved": fl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                      "frac": fl / FP64_PEAK_TFLOPS if fl else None,
                      "peak_note": "FP64 pipe, nominal 1.25 TFLOP/s (the recipe's unit rate); flops are the "
                                   "kernel's executed FP64 operations (ncu, DFMA = 2)"}
    else:
        out["implementation_bytes_per_zone_stage"] = BYTES_PER_ZONE_UPDATE_MIXED / 4.0
    out["stage_kernels"] = k.get("stage_kernels")
    if k.get("autotune"):
        out["autotune"] = k["autotune"]
    prec = 0 if r["precision"] == "fp64" else 1
    ids = k.get("kernel_ids_used") or []
    per_zone = [NCU_TRAFFIC_PER_ZONE.get((prec, i)) for i in ids]
    traffic = None
    if per_zone and None not in per_zone:  # every level on a captured kernel
        traffic = max(per_zone) * k["zones_per_launch"]
    out.update({"traffic": traffic,
                "traffic_note": "ncu DRAM bytes averaged over the four RK4 stage launches of the 96^3 patch, "
                                "per zone, times the zones of the average launch",
                "kernel": k["name"], "launch_ms": k["ms"], "launches_per_step": k["launches"] / k["steps"],
                "share_of_step": k["ms"] * k["launches"] / k["steps"] / r["ms"],
                "algorithmic_bytes_per_launch": alg})
    return out


def measure(torch, sk, h, precision, args, world, dist):
    zu = h.zone_updates_per_coarse_step()
    prm = sk.Params(courant=args.courant, precision=1 if precision == "mixed" else 0)
    stream = torch.cuda.Stream()
    g = sk.Grid(len(h.levels), h.dx0, h.patches, prm, stream=stream)
    g.set_overlap(not args.serial_ghosts)
    g.set_initial_data(1, h.masses, h.positions)
    if args.kernel is not None and precision == "mixed":
        for l in range(len(h.levels)):
            g.set_stage_kernel(l, args.kernel)
    tune = None
    if precision == "mixed" and not args.no_autotune and args.kernel is None:
        us = g.autotune(reps=3)
        tune = {"kernels": [sk.STAGE_KERNELS[g.stage_kernel(l)] for l in range(len(h.levels))],
                "us_per_launch": [[round(float(x), 1) for x in row] for row in us]}
    for _ in range(args.warmup):
        g.level_step(0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        g.level_step(0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, dist)
    norms = list(map(float, g.constraints(0)))  # also checks the state stayed finite
    nprof = max(1, min(args.steps, 2))
    kern = stage_kernel_timing(g, nprof, overlap=not args.serial_ghosts)
    kern["steps"] = nprof
    g.close()
    kern["kernel_ids_used"] = sorted(set(kern["kernel_ids"]))
    kern["stage_kernels"] = [sk.STAGE_KERNELS[k] for k in kern.pop("kernel_ids")]
    if tune:
        kern["autotune"] = tune
    out = {"precision": precision, "value": whole_job_value(zu, world, ms), "ms": ms, "kern": kern,
           "constraints_l0": norms}
    if not args.no_e2e:
        out["e2e"] = end_to_end(torch, sk, h, prm, args, world, dist)
    return out


def zsym_case(torch, sk, args):
    """The 7-level binary with equatorial reflection symmetry (Sec. 2.2.2):
    the z >= 0 half of every patch is evolved (38.9 M zone updates per coarse
    step instead of 77.8 M).  Reports zone-updates/s of the half domain and
    the full-domain equivalent (the physical domain covered per second), both
    precisions."""
    import initial_data as idd
    h = idd.upper_half_hierarchy(hierarchy())
    zu = h.zone_updates_per_coarse_step()
    out = {"case": "amr7-zsym", "zone_updates_per_step": zu, "courant": args.courant, "runs": {}}
    for name, prec in (("mixed", 1), ("fp64", 0)):
        g = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(courant=args.courant, precision=prec, zsym=1),
                    stream=torch.cuda.Stream())
        g.set_initial_data(1, h.masses, h.positions)
        if prec:
            g.autotune(reps=3)
        steps = args.steps if prec else max(1, args.steps // 2)
        for _ in range(args.warmup):
            g.level_step(0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(g.stream)
        for _ in range(steps):
            g.level_step(0)
        e1.record(g.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out["runs"][name] = {"ms_per_step": ms, "zone_updates_per_s": zu / (ms * 1e-3),
                             "full_domain_equivalent_per_s": 2 * zu / (ms * 1e-3),
                             "constraints_l0": list(map(float, g.constraints(0)))}
        g.close()
        del g
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def moving_case(torch, sk, args):
    """Moving boxes (Sec. 2.2.1) on the 7-level binary in mixed precision:
    the L5/L6 patches follow their punctures, tracked after every L6 step
    inside the captured coarse step, and sacrak_regrid runs after every coarse
    step (a host synchronisation; a patch move rebuilds the graph).  Three
    runs of --steps coarse steps each: static boxes, moving boxes with the
    data at rest (Brill-Lindquist, the punctures barely move), and moving
    boxes with a uniform shift of 0.05 added (the punctures drift by -0.05
    per unit time and the boxes follow).  CUDA events around the whole loop,
    regrids included."""
    h = hierarchy()
    zu = h.zone_updates_per_coarse_step()
    follow = [-1 if p.level < 5 else (0 if p.origin[0] + 0.5 * p.n[0] * p.dx > 0 else 1) for p in h.patches]
    out = {"case": "amr7-moving", "zone_updates_per_step": zu, "courant": args.courant, "follow": follow,
           "runs": {}}
    for name, moving, drift in (("static", False, 0.0), ("moving", True, 0.0), ("moving-drift", True, 0.05)):
        g = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(courant=args.courant, precision=1),
                    stream=torch.cuda.Stream())
        g.set_initial_data(1, h.masses, h.positions)
        if drift:
            for i in range(len(h.patches)):
                u = g.download_fields(i)
                u[19] += drift
                g.upload_fields(i, u)
        g.autotune(reps=3)
        if moving:
            g.track_punctures(h.positions, follow)
        for _ in range(args.warmup):
            g.level_step(0)
            if moving:
                g.regrid()
        moved = 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(g.stream)
        for _ in range(args.steps):
            g.level_step(0)
            if moving:
                moved += g.regrid()
        e1.record(g.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        run = {"ms_per_step": ms, "zone_updates_per_s": zu / (ms * 1e-3), "patches_moved": moved,
               "constraints_l0": list(map(float, g.constraints(0)))}
        if moving:
            run["punctures"] = g.punctures().tolist()
            run["origins_l6"] = [g.patch_origin(i) for i in range(len(h.patches)) if h.patches[i].level == 6]
        out["runs"][name] = run
        g.close()
        del g
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def psi4_case(torch, sk, args):
    """Psi4 extraction (Sec. 2.3) on the 7-level binary (mixed precision)
    after --adm-steps coarse steps: the modes l = 2..8 on spheres of levels 0
    and 1 (64 x 128 points), the GPU's time per call (CUDA events, the call
    returns the modes to the host) and the oracle's on the downloaded state
    (one host thread), their largest difference relative to the largest
    mode, and the waveform post-processing (Nakano, FFI) of a 65536-sample
    series on the GPU."""
    import initial_data as idd
    import oracle
    from oracle import waveform
    h = hierarchy()
    g = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(courant=args.courant, precision=1),
                stream=torch.cuda.Stream())
    g.set_initial_data(1, h.masses, h.positions)
    for _ in range(args.adm_steps):
        g.level_step(0)
    torch.cuda.synchronize()
    nt, nph, lmax, reps = 64, 128, 8, 10
    rows = []
    for pid, r in ((0, 100.0), (1, 40.0)):
        p = h.patches[pid]
        for _ in range(2):
            mg = g.psi4_modes(pid, (0.0, 0.0, 0.0), r, nt, nph, lmax)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(g.stream)
        for _ in range(reps):
            mg = g.psi4_modes(pid, (0.0, 0.0, 0.0), r, nt, nph, lmax)
        e1.record(g.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        u = g.download_fields(pid)
        t0 = time.perf_counter()
        mo = oracle.psi4_modes(p, u, (0.0, 0.0, 0.0), r, nt, nph, lmax)
        to = time.perf_counter() - t0
        scale = max(abs(v) for v in mo.values())
        rows.append({"patch": pid, "r": r, "gpu_ms_per_call": ms, "oracle_ms_per_call": to * 1e3,
                     "sphere_points_per_s": nt * nph / (ms * 1e-3),
                     "max_mode": scale, "psi4_22": [mg[(2, 2)].real, mg[(2, 2)].imag],
                     "max_diff_over_max_mode": max(abs(mg[k] - mo[k]) for k in mo) / scale})
    g.close()
    n = 65536
    t = np.linspace(0.0, 2000.0, n)
    psi = 1e-3 * np.exp(-1j * (0.05 * t + 1e-5 * t * t))
    wt = {}
    for name, fn in (("nakano", lambda: sk.nakano_extrapolate(t, psi, 2, 100.0, 1.0)),
                     ("ffi", lambda: sk.ffi_strain(psi, t[1] - t[0], 0.005))):
        fn()
        t0 = time.perf_counter()
        for _ in range(5):
            fn()
        wt[name + "_ms_per_call_incl_transfers"] = (time.perf_counter() - t0) / 5 * 1e3
    t0 = time.perf_counter()
    waveform.nakano_extrapolate(t, psi, 2, 100.0, 1.0)
    wt["nakano_oracle_ms"] = (time.perf_counter() - t0) * 1e3
    print(json.dumps({"case": "psi4", "coarse_steps": args.adm_steps, "ntheta": nt, "nphi": nph, "lmax": lmax,
                      "rows": rows, "waveform_65536": wt}), flush=True)


def adm_case(torch, sk, args):
    """ADM mass, J_z and linear momentum (Sec. 2.3, Sec. 3.2) on coordinate
    spheres of the 7-level binary (mixed precision) after --adm-steps coarse
    steps: the GPU's values, the oracle's on the downloaded state, and the
    time per call of the GPU integral (64 x 128 sphere points; CUDA events on
    the grid's stream, the call returns its five numbers to the host) next to
    the oracle's time on the host cores.  Brill-Lindquist data: M -> m1 + m2
    = 1 as r grows, J_z = P = 0."""
    import initial_data as idd
    import oracle
    h = hierarchy()
    g = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(courant=args.courant, precision=1),
                stream=torch.cuda.Stream())
    g.set_initial_data(1, h.masses, h.positions)
    for _ in range(args.adm_steps):
        g.level_step(0)
    torch.cuda.synchronize()
    nt, nph, reps = 64, 128, 20
    rows = []
    for pid, r in ((0, 100.0), (0, 150.0), (1, 40.0), (1, 80.0)):
        p = h.patches[pid]
        for _ in range(3):
            vg = g.adm_integrals(pid, (0.0, 0.0, 0.0), r, nt, nph)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(g.stream)
        for _ in range(reps):
            vg = g.adm_integrals(pid, (0.0, 0.0, 0.0), r, nt, nph)
        e1.record(g.stream)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / reps
        ms = e0.elapsed_time(e1) / reps
        u = g.download_fields(pid)
        t0 = time.perf_counter()
        vo = oracle.adm_integrals(p, u, (0.0, 0.0, 0.0), r, nt, nph)
        to = time.perf_counter() - t0
        scale = max(abs(v) for v in vo)
        rows.append({"patch": pid, "level": p.level, "dx": p.dx, "r": r, "gpu": list(vg), "oracle": list(vo),
                     "max_abs_diff_over_max": max(abs(a - b) for a, b in zip(vg, vo)) / scale,
                     "gpu_ms_per_call": ms, "gpu_wall_ms_per_call": wall * 1e3,
                     "sphere_points_per_s": nt * nph / (ms * 1e-3), "oracle_ms_per_call": to * 1e3,
                     "oracle_threads": 1})
    print(json.dumps({"case": "adm", "coarse_steps": args.adm_steps, "time": g.level_time(0),
                      "ntheta": nt, "nphi": nph, "rows": rows}), flush=True)
    g.close()


def _gw_grid(torch, sk, n, precision, **prm):
    """Periodic unit box [-1/2, 1/2]^3 with n^3 cells, harmonic slicing,
    frozen shift, Courant 0.25 (the gauge-wave / robust-stability setup)."""
    import initial_data as idd
    p = idd.centred_patch(n, 1.0 / n)
    g = sk.Grid(1, p.dx, [p], sk.Params(lapse=1, shift=1, bc=1, courant=0.25, precision=precision),
                stream=torch.cuda.Stream())
    return p, g


def gauge_wave_case(torch, sk, args):
    """Gauge wave A = 0.01, wavelength = box size 1, on periodic 3D grids of
    32^3, 64^3 and 128^3 cells: 1000 RK4 steps at 32^3 and the same final time
    t = 1000 * 0.25 / 32 on the finer grids (2000 and 4000 steps).  Reports
    the max-norm error against the closed form per resolution, the
    convergence rates, the constraint norms and the wall time."""
    import initial_data as idd
    sizes = [int(x) for x in args.sizes.split(",")]
    steps0 = args.gw_steps
    t_final = steps0 * 0.25 / sizes[0]
    out = {"case": "gauge-wave", "amp": 0.01, "wavelength": 1.0, "courant": 0.25, "t_final": t_final,
           "precision": args.precision if args.precision != "both" else "fp64", "runs": []}
    prec = 1 if out["precision"] == "mixed" else 0
    errs = []
    for n in sizes:
        p, g = _gw_grid(torch, sk, n, prec)
        g.set_initial_data(2, gw_amp=0.01, gw_len=1.0)
        nsteps = steps0 * n // sizes[0]
        h0 = g.constraints(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = []
        for s in range(nsteps):
            g.rk4_step(0)
            if (s + 1) % (nsteps // 4) == 0:
                hist.append([s + 1] + list(map(float, g.constraints(0))))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        u = g.download_fields(0)[:, 3:-3, 3:-3, 3:-3]
        ex = idd.gauge_wave(p, 0.01, t=g.level_time(0))[:, 3:-3, 3:-3, 3:-3]
        e = np.abs(u - ex).max(axis=(1, 2, 3))
        errs.append(float(e.max()))
        out["runs"].append({"n": n, "steps": nsteps, "t": g.level_time(0), "max_err": float(e.max()),
                            "max_err_per_field": {k: float(v) for k, v in zip(idd.FIELD_NAMES, e) if v > 0},
                            "constraints_t0": list(map(float, h0)), "constraints_history": hist,
                            "wall_s": wall, "zone_updates_per_s": n ** 3 * nsteps / wall})
        g.close()
    out["rates"] = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    print(json.dumps(out), flush=True)


def robust_stability_case(torch, sk, args):
    """Minkowski plus uniform noise of amplitude 1e-10 (dx/dx0)^2, dx0 = 1/32,
    on periodic 32^3, 64^3, 128^3 grids, 1000 RK4 steps each (Courant 0.25,
    harmonic slicing, frozen shift); the Hamiltonian and momentum constraint
    norms every 100 steps."""
    import initial_data as idd
    sizes = [int(x) for x in args.sizes.split(",")]
    out = {"case": "robust-stability", "courant": 0.25, "steps": args.gw_steps,
           "precision": args.precision if args.precision != "both" else "fp64", "runs": []}
    prec = 1 if out["precision"] == "mixed" else 0
    for n in sizes:
        p, g = _gw_grid(torch, sk, n, prec)
        amp = 1e-10 * (32.0 / n) ** 2
        g.set_initial_data(0, noise_amp=amp, seed=idd.STABILITY_SEED)
        flat = idd.minkowski(p)[:, 3:-3, 3:-3, 3:-3]

        def dev():
            d = np.abs(g.download_fields(0)[:, 3:-3, 3:-3, 3:-3] - flat)
            return [float(x) for x in d.max(axis=(1, 2, 3))]

        hist = [[0] + list(map(float, g.constraints(0)))]
        devs = [[0] + dev()]
        for s in range(args.gw_steps):
            g.rk4_step(0)
            if (s + 1) % 100 == 0:
                hist.append([s + 1] + list(map(float, g.constraints(0))))
                devs.append([s + 1] + dev())
        out["runs"].append({"n": n, "noise_amp": amp, "t": g.level_time(0), "constraints_history": hist,
                            "field_names": idd.FIELD_NAMES, "max_dev_from_flat_history": devs,
                            "growth_H": hist[-1][1] / hist[0][1] if hist[0][1] > 0 else None})
        g.close()
    print(json.dumps(out), flush=True)


def _time_rk4(torch, g, level, steps, warm=1):
    for _ in range(warm):
        g.rk4_step(level)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(g.stream)
    for _ in range(steps):
        g.rk4_step(level)
    e1.record(g.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def sweep_case(torch, sk, args):
    """Large-AMR throughput sweep.  (a) Single patches of 48^3 .. 192^3
    (Brill-Lindquist m = 1 at the centre, Sommerfeld ghosts): the autotuned
    mixed-precision stage kernel and the FP64 kernel, zone updates/s of RK4
    steps and the HBM fraction.  (b) The 10-level hierarchy (L0-L5 one 192^3
    patch, L6-L9 two 160^3 patches around m = 0.6 / 0.4 punctures): per level,
    the zone updates/s of one RK4 step of that level (its ghost fills
    included) in both precisions, and one full coarse step (1023 level steps,
    one CUDA graph) in mixed precision."""
    import initial_data as idd
    hbm = float(_peaks().get("hbm_gbs", 6800.0))
    out = {"case": "amr10-sweep", "hbm_gbs": hbm, "courant": args.courant, "patches": [], "levels": []}
    for n in [int(x) for x in args.sweep_sizes.split(",")]:
        p = idd.centred_patch(n, 16.0 / n)
        row = {"n": n}
        for prec in (1, 0):
            g = sk.Grid(1, p.dx, [p], sk.Params(courant=args.courant, precision=prec), stream=torch.cuda.Stream())
            g.set_initial_data(1, [1.0], [(0.0, 0.0, 0.0)])
            key = "mixed" if prec else "fp64"
            if prec:
                us = g.autotune(reps=3, use_cache=False)[0]
                row["autotune_us_per_stage1"] = [round(float(x), 1) for x in us]
                row["kernel"] = sk.STAGE_KERNELS[g.stage_kernel(0)]
            ms = _time_rk4(torch, g, 0, 5 if prec else 2)
            zu = p.active_points / (ms * 1e-3)
            bpz = BYTES_PER_ZONE_UPDATE
            row[key] = {"ms_per_rk4_step": ms, "zone_updates_per_s": zu, "hbm_frac": zu * bpz / (hbm * 1e9)}
            g.close()
            del g
            torch.cuda.empty_cache()
        out["patches"].append(row)
        print(json.dumps(row), flush=True)
    h = idd.binary_10_level()
    for prec in (1, 0):
        prm = sk.Params(courant=args.courant, precision=prec)
        need = sk.arena_bytes(len(h.levels), h.patches, prm)
        free, total = torch.cuda.mem_get_info()
        key = "mixed" if prec else "fp64"
        if need > free - (8 << 30):
            out["levels"].append({key: "skipped: arena %.1f GB, free %.1f GB" % (need / 1e9, free / 1e9)})
            continue
        g = sk.Grid(len(h.levels), h.dx0, h.patches, prm, stream=torch.cuda.Stream())
        g.set_initial_data(1, h.masses, h.positions)
        res = {"precision": key, "arena_gb": need / 1e9, "per_level": []}
        if prec:
            g.autotune(reps=2)
        for l, lv in enumerate(h.levels):
            act = sum(p.active_points for p in lv)
            ms = _time_rk4(torch, g, l, 2)
            zu = act / (ms * 1e-3)
            bpz = BYTES_PER_ZONE_UPDATE
            res["per_level"].append({"level": l, "patches": [list(p.n) for p in lv],
                                     "kernel": sk.STAGE_KERNELS[g.stage_kernel(l)],
                                     "ms_per_rk4_step": ms, "zone_updates_per_s": zu,
                                     "hbm_frac": zu * bpz / (hbm * 1e9)})
        if prec and not args.no_coarse:
            # the RK4 steps above advanced the levels independently: start the
            # coarse step from fresh data
            g.set_initial_data(1, h.masses, h.positions)
            g.level_step(0)  # records the graph
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(g.stream)
            g.level_step(0)
            e1.record(g.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            zu = h.zone_updates_per_coarse_step()
            res["coarse_step"] = {"ms": ms, "zone_updates": zu, "zone_updates_per_s": zu / (ms * 1e-3),
                                  "hbm_frac": zu / (ms * 1e-3) * BYTES_PER_ZONE_UPDATE / (hbm * 1e9),
                                  "constraints_l0": list(map(float, g.constraints(0)))}
        out["levels"].append(res)
        print(json.dumps(res), flush=True)
        g.close()
        del g
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def tov_case(torch, sk, args):
    """The coupled RK4 step of spacetime and fluid (Sec. 2.1.2, 2.2) for a TOV
    star (cold Gamma = 2 polytrope, K = 100, rho_c = 1.28e-3, M = 1.40,
    Gamma_th = 1.8) on one FP64 patch of n^3 cells over [-16, 16]^3: 1+log
    slicing and Gamma driver, Sommerfeld ghosts for the spacetime, outflow
    ghosts for the fluid, atmosphere 1e-12 rho_c.  Each step is one captured
    graph replay (the RK4 step and the level bookkeeping).  Reported: zone
    updates/s of the coupled step and of the spacetime alone on the same
    patch, and the drift of the central density over the timed steps."""
    import initial_data as idd
    from initial_data.tov import TOV, tov_patch_data
    n = args.tov_n
    p = idd.centred_patch(n, 32.0 / n)
    star = TOV()
    rho_atm, r_atm = 1e-12 * 1.28e-3, 8 * 32.0
    u, prim = tov_patch_data(p, star, rho_atm)
    c = p.g + n // 2
    out = {"case": "tov", "n": n, "dx": p.dx, "courant": args.courant, "zones": p.active_points,
           "star": {"M": star.M, "R_areal": star.R, "R_isotropic": star.Rbar}, "runs": {}}
    for name, matter in (("spacetime+fluid", 1), ("spacetime", 0)):
        g = sk.Grid(1, p.dx, [p], sk.Params(courant=args.courant, matter=matter), stream=torch.cuda.Stream())
        if matter:
            g.set_eos(star.K, [star.G], (), 1.8)
            g.set_atmosphere(rho_atm, r_atm)
        g.upload_fields(0, u)
        if matter:
            g.upload_matter(0, prim)
        for _ in range(args.warmup):
            g.level_step(0)
        rho0 = float(g.download_matter(0)[0, c, c, c]) if matter else None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(g.stream)
        for _ in range(args.steps):
            g.level_step(0)
        e1.record(g.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        run = {"ms_per_rk4_step": ms, "zone_updates_per_s": p.active_points / (ms * 1e-3),
               "constraints": list(map(float, g.constraints(0)))}
        if matter:
            rho1 = float(g.download_matter(0)[0, c, c, c])
            run["central_density_drift"] = (rho1 - rho0) / rho0
        out["runs"][name] = run
        g.close()
        del g
        torch.cuda.empty_cache()
    r = out["runs"]
    out["fluid_ms_per_step"] = r["spacetime+fluid"]["ms_per_rk4_step"] - r["spacetime"]["ms_per_rk4_step"]
    print(json.dumps(out), flush=True)


def _rest_mass(patches, fields, prims, children):
    """Total rest mass of the composite grid, sum of sqrt(gamma) rho w dV over
    the active cells not covered by a child (sqrt(gamma) = sqrt(det gt) / W^3,
    w = sqrt(1 + gamma^ij u_i u_j), gamma^ij = W^2 gt^ij)."""
    total = 0.0
    for pid, (p, u, pr) in enumerate(zip(patches, fields, prims)):
        g = p.g
        a = (slice(g, -g),) * 3
        W = u[0][a]
        gt = [u[1 + c][a] for c in range(6)]
        gxx, gxy, gxz, gyy, gyz, gzz = gt
        det = gxx * (gyy * gzz - gyz * gyz) - gxy * (gxy * gzz - gyz * gxz) + gxz * (gxy * gyz - gyy * gxz)
        inv = [(gyy * gzz - gyz * gyz), (gxz * gyz - gxy * gzz), (gxy * gyz - gxz * gyy),
               (gxx * gzz - gxz * gxz), (gxy * gxz - gxx * gyz), (gxx * gyy - gxy * gxy)]
        ul = [pr[2 + d][a] for d in range(3)]
        pairs = [(0, 0, 0), (0, 1, 1), (0, 2, 2), (1, 1, 3), (1, 2, 4), (2, 2, 5)]
        uu = sum((1.0 if i == j else 2.0) * inv[c] * ul[i] * ul[j] for i, j, c in pairs) / det * W * W
        D = np.sqrt(det) / W ** 3 * pr[0][a] * np.sqrt(1.0 + uu)
        for cid in children[pid]:
            c = patches[cid]
            off = [int(round((c.origin[d] - p.origin[d]) / p.dx)) for d in range(3)]
            D[off[2]:off[2] + c.n[2] // 2, off[1]:off[1] + c.n[1] // 2, off[0]:off[0] + c.n[0] // 2] = 0.0
        total += float(D.sum()) * p.dx ** 3
    return total


def tov_amr_case(torch, sk, args):
    """The coupled coarse step of spacetime and fluid (Sec. 2.1.2, 2.2,
    2.2.1) for the TOV star of the `tov` case on two levels: a 96^3 patch at
    dx = 1/2 over [-24, 24]^3 and a 96^3 child at dx = 1/4 over [-12, 12]^3
    around the star (R = 8.1 isotropic), the fluid's ghosts at the refinement
    boundary by WENO5 / Lagrange prolongation, restriction and reflux after
    the child's two steps.  Each step is one captured graph replay.
    Reported: zone updates/s of the coupled coarse step (3 x 96^3 zone
    updates) and of the spacetime alone on the same hierarchy, and the
    relative change of the total rest mass over the timed steps (outflow
    through the atmosphere at the outer boundary and atmosphere resets only:
    the refinement boundary conserves it)."""
    import initial_data as idd
    from initial_data.tov import TOV, tov_patch_data
    star = TOV()
    P0 = idd.Patch(n=(96, 96, 96), dx=0.5, origin=(-24.0, -24.0, -24.0), level=0)
    C1 = idd.Patch(n=(96, 96, 96), dx=0.25, origin=(-12.0, -12.0, -12.0), level=1)
    ps = [P0, C1]
    rho_atm, r_atm = 1e-12 * 1.28e-3, 8 * 24.0
    data = [tov_patch_data(p, star, rho_atm) for p in ps]
    zu = P0.active_points + 2 * C1.active_points
    out = {"case": "tov-amr", "levels": [{"n": p.n[0], "dx": p.dx} for p in ps], "courant": args.courant,
           "zone_updates_per_step": zu, "star": {"M": star.M, "R_isotropic": star.Rbar}, "runs": {}}
    for name, matter in (("spacetime+fluid", 1), ("spacetime", 0)):
        g = sk.Grid(2, P0.dx, ps, sk.Params(courant=args.courant, matter=matter), stream=torch.cuda.Stream())
        if matter:
            g.set_eos(star.K, [star.G], (), 1.8)
            g.set_atmosphere(rho_atm, r_atm)
        for i, (u, prim) in enumerate(data):
            g.upload_fields(i, u)
            if matter:
                g.upload_matter(i, prim)
        for _ in range(args.warmup):
            g.level_step(0)
        if matter:
            m0 = _rest_mass(ps, [g.download_fields(i) for i in range(2)], [g.download_matter(i) for i in range(2)],
                            [[1], []])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(g.stream)
        for _ in range(args.steps):
            g.level_step(0)
        e1.record(g.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        run = {"ms_per_coarse_step": ms, "zone_updates_per_s": zu / (ms * 1e-3)}
        if matter:
            m1 = _rest_mass(ps, [g.download_fields(i) for i in range(2)], [g.download_matter(i) for i in range(2)],
                            [[1], []])
            run["rest_mass_change"] = (m1 - m0) / m0
        out["runs"][name] = run
        g.close()
        del g
        torch.cuda.empty_cache()
    r = out["runs"]
    out["fluid_ms_per_step"] = r["spacetime+fluid"]["ms_per_coarse_step"] - r["spacetime"]["ms_per_coarse_step"]
    print(json.dumps(out), flush=True)


def tov_moving_case(torch, sk, args):
    """Neutron-star tracking with moving fluid patches (Sec. 2.2.1) on the
    tov-amr hierarchy: the star centred at x = 3.1, the child (centred on
    the origin) following its density maximum.  After the warm-up steps the
    first regrid shifts the child by trunc(3.125 / 0.5) = 6 parent cells
    (the fluid moved with copy and conservative prolongation, caches and
    graph rebuilt; wall time of the synchronous call); then --steps coarse
    steps each followed by a regrid (CUDA events around the loop, the
    regrids' density maximum and host synchronisation included) and --steps
    without.  Reported: the times, the child's origins, and the relative
    rest-mass change across the move (the WENO fallback next to the star's
    surface makes it non-zero) and over the steps."""
    import dataclasses
    import initial_data as idd
    from initial_data.tov import TOV, tov_patch_data
    star = TOV()
    P0 = idd.Patch(n=(96, 96, 96), dx=0.5, origin=(-24.0, -24.0, -24.0), level=0)
    C1 = idd.Patch(n=(96, 96, 96), dx=0.25, origin=(-12.0, -12.0, -12.0), level=1)
    ps = [P0, C1]
    rho_atm, r_atm = 1e-12 * 1.28e-3, 8 * 24.0
    data = [tov_patch_data(p, star, rho_atm, centre=(3.1, 0.0, 0.0)) for p in ps]
    zu = P0.active_points + 2 * C1.active_points
    g = sk.Grid(2, P0.dx, ps, sk.Params(courant=args.courant, matter=1), stream=torch.cuda.Stream())
    g.set_eos(star.K, [star.G], (), 1.8)
    g.set_atmosphere(rho_atm, r_atm)
    for i, (u, prim) in enumerate(data):
        g.upload_fields(i, u)
        g.upload_matter(i, prim)
    g.track_stars([-1, 0])

    def mass():
        geo = [P0, dataclasses.replace(C1, origin=g.patch_origin(1))]
        return _rest_mass(geo, [g.download_fields(i) for i in range(2)], [g.download_matter(i) for i in range(2)],
                          [[1], []])
    for _ in range(args.warmup):
        g.level_step(0)
    torch.cuda.synchronize()
    m0 = mass()
    star_before = g.density_maximum(1)
    t0 = time.perf_counter()
    moved = g.regrid()
    move_ms = (time.perf_counter() - t0) * 1e3
    m1 = mass()
    out = {"case": "tov-moving", "zone_updates_per_step": zu, "courant": args.courant,
           "star_before": star_before, "first_regrid": {"patches_moved": moved, "wall_ms": move_ms,
                                                        "origin_l1": g.patch_origin(1),
                                                        "rest_mass_change": (m1 - m0) / m0},
           "runs": {}}
    for name, regrid in (("regrid every step", True), ("no regrid", False)):
        n = 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(g.stream)
        for _ in range(args.steps):
            g.level_step(0)
            if regrid:
                n += g.regrid()
        e1.record(g.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out["runs"][name] = {"ms_per_coarse_step": ms, "zone_updates_per_s": zu / (ms * 1e-3), "patches_moved": n}
    out["rest_mass_change_over_steps"] = (mass() - m1) / m1
    out["star_after"] = g.density_maximum(1)
    g.close()
    print(json.dumps(out), flush=True)


def uniform_case(torch, sk, args):
    """RK4 steps of the level-0 96^3 patch alone (Sommerfeld ghosts): the
    small, single-kernel case used for ncu captures."""
    import initial_data as idd
    h = hierarchy()
    p = h.levels[0][0]
    prm = sk.Params(courant=args.courant, precision=1 if args.precision == "mixed" else 0)
    stream = torch.cuda.Stream()
    g = sk.Grid(1, p.dx, [p], prm, stream=stream)  # (--precision both runs FP64 here)
    g.set_initial_data(1, h.masses, h.positions)
    tune = None
    if prm.precision == 1:
        if not args.no_autotune:
            tune = [round(float(x), 1) for x in g.autotune(reps=3, use_cache=False)[0]]
        if args.kernel is not None:
            g.set_stage_kernel(0, args.kernel)
    for _ in range(args.warmup):
        g.rk4_step(0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        g.rk4_step(0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    g.constraints(0)
    print(json.dumps({"case": "uniform96", "ms_per_rk4_step": ms,
                      "zone_updates_per_s": p.active_points / (ms * 1e-3),
                      "stage_kernel": sk.STAGE_KERNELS[g.stage_kernel(0)],
                      "autotune_us_per_stage1_launch": tune}), flush=True)
    g.close()


def mixed_error_case(torch, sk, args):
    """Evolve the 7-level binary in FP64 and in mixed precision from the same
    data for --coarse-steps coarse steps; report per level and field the
    max |mixed - FP64| (absolute and over the field's max |FP64|) and both
    runs' constraint norms.  --error-kernels lists the mixed stage kernels to
    compare (one mixed run each, default: the default kernel).  --fp64-twin
    adds an FP64 run from the same data perturbed by 1e-7 relative, the size
    of FP32 rounding: how far two FP64 evolutions part from differences of
    that size, beside how far mixed and FP64 part."""
    import initial_data as idd
    h = hierarchy()
    grids = {}
    kernels = [int(k) for k in args.error_kernels.split(",")] if args.error_kernels else [None]
    runs = [("fp64", 0, None)] + [("mixed" if k is None else "mixed-k%d" % k, 1, k) for k in kernels]
    if args.fp64_twin:
        runs.append(("fp64-perturbed", 0, None))
    for name, prec, k in runs:
        g = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(courant=args.courant, precision=prec),
                    stream=torch.cuda.Stream())
        g.set_initial_data(1, h.masses, h.positions)
        if name == "fp64-perturbed":
            # every value times (1 + 1e-7 r), r uniform in [-1, 1): the size of
            # the FP32 rounding of the mixed path's arithmetic, in FP64
            for i, p in enumerate(h.patches):
                u = g.download_fields(i)
                r = idd.add_noise(p, np.zeros_like(u), 1.0, 987654321, idd.level_origin(h, p.level))
                g.upload_fields(i, u * (1.0 + 1e-7 * r))
        if k is not None:
            for l in range(len(h.levels)):
                g.set_stage_kernel(l, k)
        grids[name] = g
    times = {}
    for name, g in grids.items():
        t0 = time.perf_counter()
        for _ in range(args.coarse_steps):
            g.level_step(0)
        torch.cuda.synchronize()
        times[name] = (time.perf_counter() - t0) / args.coarse_steps
    report = {"case": "mixed-error", "coarse_steps": args.coarse_steps, "courant": args.courant,
              "t_final": grids["fp64"].level_time(0),
              "s_per_coarse_step": times, "stage_kernels": {n: sk.STAGE_KERNELS[grids[n].stage_kernel(0)]
                                                            for n in grids}, "levels": []}
    for l in range(len(h.levels)):
        ids = [i for i, p in enumerate(h.patches) if p.level == l]
        row = {"level": l, "constraints_fp64": list(map(float, grids["fp64"].constraints(l)))}
        for name in grids:
            if name == "fp64":
                continue
            err = np.zeros(25)
            rel = np.zeros(25)
            for i in ids:
                a = grids["fp64"].download_fields(i)[:, 3:-3, 3:-3, 3:-3]
                m = grids[name].download_fields(i)[:, 3:-3, 3:-3, 3:-3]
                d = np.abs(m - a).max(axis=(1, 2, 3))
                sc = np.abs(a).max(axis=(1, 2, 3))
                err = np.maximum(err, d)
                rel = np.maximum(rel, np.where(sc > 0, d / np.where(sc > 0, sc, 1), d))
            sfx = "" if name == "mixed" else "_" + name
            row["max_abs_err" + sfx] = {n: float(v) for n, v in zip(idd.FIELD_NAMES, err)}
            row["max_rel_err" + sfx] = {n: float(v) for n, v in zip(idd.FIELD_NAMES, rel)}
            row["constraints_" + name] = list(map(float, grids[name].constraints(l)))
        report["levels"].append(row)
    print(json.dumps(report), flush=True)
    for g in grids.values():
        g.close()


def stage_kernel_timing(g, steps, overlap=True):
    """Average duration of one launch of the fused RHS + RK4 stage kernel over
    `steps` coarse steps, from CUDA events bracketing every launch on the
    grid's stream (eager launches while profiling is on).  This pass runs the
    serial ghost schedule, so that no ghost fill shares the SMs with the
    bracketed kernel; `overlap` is the schedule restored afterwards."""
    ids = [g.stage_kernel(l) for l in range(g.nlevels)]
    g.set_overlap(False)
    g.profile_enable(True)
    for _ in range(steps):
        g.level_step(0)
    ms, n, zones = g.profile_read()
    g.profile_enable(False)
    g.set_overlap(overlap)
    per = ms / n
    zones_per_launch = zones / n
    fz = FLOPS_PER_ZONE_STAGE.get(g.params.precision)
    if g.params.precision == 0:
        name = "z4c_stage_fp64_kernel"
    else:
        import paper_2607_08743_gb300 as sk
        kn = {0: "z4c_stage_mixed_kernel"}
        kn.update({k: "z4c_stage_tma_kernel (%s)" % sk.STAGE_KERNELS[k] for k in (1, 2, 3, 4)})
        kn.update({k: "z4c_stage_ldg_kernel (%s)" % sk.STAGE_KERNELS[k] for k in (5, 6, 8, 9, 10, 11, 12, 13, 14, 18)})
        kn.update({k: "z4c_stage_pair_kernel (%s)" % sk.STAGE_KERNELS[k] for k in (15, 16, 17)})
        kn.update({k: "z4c_stage_fixed_kernel (%s)" % sk.STAGE_KERNELS[k] for k in (19, 20)})
        kn[7] = "z4c_deriv_kernel + z4c_algebra_kernel"
        names = sorted({kn[k] for k in ids})
        name = " + ".join(names)
    return {"name": name, "kernel_ids": ids,
            "ms": per, "launches": n, "share_of_step": None,
            "bytes_per_launch": zones_per_launch * ALG_BYTES_PER_ZONE_STAGE,
            "flops_per_launch": zones_per_launch * fz if fz else None,
            "traffic": None, "zones_per_launch": zones_per_launch}


# FP64 flops per zone per stage of the fused kernel (DFMA counted as 2), from
# the ncu instruction counts of one launch divided by the zones it updates
FLOPS_PER_ZONE_STAGE = {0: 4812}


def _gpu_local_cpus(torch):
    """The host CPUs (of those this process may use) attached to the
    current GPU's NUMA node, from sysfs; None where that is unknown."""
    try:
        pr = torch.cuda.get_device_properties(torch.cuda.current_device())
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        text = open("/sys/bus/pci/devices/%s/local_cpulist" % bus).read().strip()
        cpus = set()
        for part in text.split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        local = cpus & os.sched_getaffinity(0)
        return local or None
    except Exception:
        return None


def end_to_end(torch, sk, h, prm, args, world, dist):
    """Same metric through the public API with host buffers: every step
    uploads every patch from pinned host memory, runs the coarse step and
    downloads every patch."""
    stream = torch.cuda.Stream()
    g = sk.Grid(len(h.levels), h.dx0, h.patches, prm, stream=stream)
    g.set_overlap(not args.serial_ghosts)
    g.set_initial_data(1, h.masses, h.positions)
    # the pinned host buffers on the GPU's own NUMA node (the host thread
    # runs there while it allocates and drives them), as a caller would place
    # them; the affinity is restored afterwards
    saved = os.sched_getaffinity(0)
    local = _gpu_local_cpus(torch)
    if local and local != saved:
        os.sched_setaffinity(0, local)
    host = [torch.empty(g.shape(i), dtype=torch.float64).pin_memory() for i in range(len(h.patches))]
    for i in range(len(h.patches)):
        g.download_fields(i, host[i])
    nbytes = sum(x.numel() * 8 for x in host)

    phase = [0.0, 0.0, 0.0]  # upload, coarse step, download (host clock)

    def step():
        t = time.perf_counter()
        for i in range(len(h.patches)):
            g.upload_fields(i, host[i])  # (each call synchronises)
        t1 = time.perf_counter()
        g.level_step(0)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        for i in range(len(h.patches)):
            g.download_fields(i, host[i])
        t3 = time.perf_counter()
        phase[0] += t1 - t
        phase[1] += t2 - t1
        phase[2] += t3 - t2

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    phase[:] = [0.0, 0.0, 0.0]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    ms = max_over_ranks(ms, dist)
    g.close()
    del host
    os.sched_setaffinity(0, saved)
    zu = h.zone_updates_per_coarse_step()
    return {"value": whole_job_value(zu, world, ms), "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "host_buffers": ("pinned, allocated and driven from the %d CPUs local to the GPU" % len(local)
                             if local and local != saved else "pinned (GPU-local CPUs unknown or all local)"),
            "d2h_bytes_per_step": nbytes, "ms_per_step": ms,
            "phases_ms": {"upload": 1e3 * phase[0] / args.steps, "coarse_step": 1e3 * phase[1] / args.steps,
                          "download": 1e3 * phase[2] / args.steps}}


if __name__ == "__main__":
    main()
