#!/usr/bin/env python
"""Throughput benchmark of the GB300 ghost-cell multigrid.

Metric: unknowns (|Omega_h| + |Gamma_h|) solved per second from u = 0 to
relative residual 1e-10 (||r||_inf / ||r0||_inf, r0 = (f, g)).  One step is
one whole solve of the workload with f and g already resident in HBM; an L2
flush (a 256 MB write) separates steps.  The default workload is the largest
single-GPU configuration, the 3D torus on 513^3 nodes (FP32 cycles inside
FP64 refinement), with the plain FP64 GPU solve of the same workload beside
it.  `e2e` repeats the measurement through the host-buffer entry point (host
-> device copies of f and g and the device -> host copy of u inside the
timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config torus513]
                    [--precision mixed|fp64] [--impl gcmg|reference]

Under torchrun every rank solves its own replica (the single-grid solve does
not shard); value = all ranks' unknowns / the slowest rank's time.
`--impl reference` times the FP64 CPU oracle (the correctness reference) on
bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1111_0983_gb300 import inputs  # noqa: E402

METRIC = "unknowns/s to rel. residual 1e-10"
FP64_FLOOR_NOTE = ("rel. residual ||r||/||(f,g)|| cannot go below ~2e-10 at 4097^2 in FP64 "
                   "(u rounding x 8/h^2 vs max|f|), so that grid is timed to 1e-9")
WORKLOADS = {
    # name: (problem factory, n, n_coarse, description)
    "flower4097": (inputs.flower, 4097, 33, "2D flower r-0.5-0.15 sin(5 theta), mixed D/N, 4097^2"),
    "flower1025": (inputs.flower, 1025, 33, "2D flower r-0.5-0.15 sin(5 theta), mixed D/N, 1025^2"),
    "disk65": (inputs.disk, 65, 17, "2D disk r=0.7, Dirichlet, 65^2"),
    "torus257": (inputs.torus, 257, 17, "3D torus R=0.5 r=0.25, mixed D/N, 257^3"),
    "torus513": (inputs.torus, 513, 17, "3D torus R=0.5 r=0.25, mixed D/N, 513^3"),
    "stars256": (None, None, 33, "256 seeded 2D stars, n in {129,257,513,1025}, mixed D/N, one batched solve"),
}
L2_FLUSH_BYTES = 256 << 20
# plain FP64 stalls above 1e-10 on the finest grids: the rounding of u in the
# FP64 smoother, times the 2d/h^2 of an interior row, keeps the defect of its
# iterates near these fractions of ||(f, g)|| (FP32 cycles inside FP64
# refinement only add small corrections to u and go lower); the plain FP64
# comparison is timed to these targets there
FP64_FLOOR_RTOL = {"torus513": 5e-10, "flower4097": 1e-9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="torus513", choices=sorted(WORKLOADS))
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--also", default="flower1025:1e-10,flower4097:1e-9,torus257:1e-10",
                    help="comma-separated secondary workload:rtol pairs measured after the main one ('' to skip)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--gamma", type=int, default=1)
    ap.add_argument("--impl", default="gcmg", choices=["gcmg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=256, help="domains of the batched secondary / stars256 run")
    ap.add_argument("--batch-profile", action="store_true",
                    help="after the batch measurement, one more batch solve as plain launches between "
                         "profiler start and stop (for ncu --profile-from-start off)")
    ap.add_argument("--sweep3d", type=int, default=-1,
                    help="3D interior sweep kernel (gcmg_set_sweep3d; -1: the library's default)")
    ap.add_argument("--boundary3d", type=int, default=-1,
                    help="3D boundary relaxation launch mode (gcmg_set_boundary3d; -1: the library's default)")
    ap.add_argument("--fp64", type=int, default=1,
                    help="time the plain FP64 solve of the workload beside the mixed form (1) or not (0)")
    ap.add_argument("--profile-solve", action="store_true",
                    help="after the measurement, one more solve of the workload as plain launches between "
                         "profiler start and stop (for ncu --profile-from-start off)")
    ap.add_argument("--cpu-sample-cycles", type=int, default=1)
    ap.add_argument("--cpu-single", type=int, default=1,
                    help="also time the oracle's sample on one host core (1) or not (0)")
    ap.add_argument("--paper", default="flower1025",
                    help="workload of the paper's-method comparison (junction relaxation off, V and W; '' to skip)")
    ap.add_argument("--learned", type=int, default=8,
                    help="held-out 513^2 star problems for the learned-guess comparison (0 to skip)")
    ap.add_argument("--fmg", default="flower1025",
                    help="workload of the full-multigrid comparison (plain FP64; '' to skip)")
    ap.add_argument("--write-traffic", nargs=3, metavar=("CSV", "KERNEL_REGEX", "KEY"),
                    help="record in profiles/traffic.json, under KEY, the mean DRAM bytes per launch of the "
                         "kernels matching KERNEL_REGEX in an ncu CSV (dram__bytes_read.sum, "
                         "dram__bytes_write.sum) and exit; a regex ending in '@largest' keeps only the "
                         "launches with the largest grid (the fine level)")
    ap.add_argument("--traffic-group", type=int, default=1,
                    help="with --write-traffic: bytes of a unit of this many consecutive launches (2 for the 3D "
                         "interior sweep, whose red and black half-sweeps are two launches)")
    return ap.parse_args()


def dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------- clock sampling
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


KERNEL_SOURCES = ("kernels.cu", "kernels_dev.cuh", "gcmg_internal.h")


def kernels_sha():
    """Hash of the per-level kernels' device sources, comments and
    whitespace removed (an edited comment does not invalidate a capture)."""
    import re
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1111_0983_gb300", "csrc", name)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def traffic_for(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    sources are unchanged since it was captured."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh).get(kernel_key)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    return rec.get("dram_bytes_per_launch") if rec.get("kernels_sha") == kernels_sha() else None


def write_traffic(csv_path, kernel_regex, key, group=1):
    """Mean dram__bytes_read.sum + dram__bytes_write.sum per launch of the
    matching kernels in an ncu --csv log (times `group`: the bytes of a unit
    of that many launches), into profiles/traffic.json."""
    import csv
    import re
    per, grid = {}, {}
    largest = kernel_regex.endswith("@largest")
    pattern = kernel_regex[:-len("@largest")] if largest else kernel_regex
    with open(csv_path) as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    rows = list(csv.reader(lines))
    head = rows[0]
    ci, cn, cm, cv, cu, cg = (head.index(k) for k in ("ID", "Kernel Name", "Metric Name", "Metric Value",
                                                        "Metric Unit", "Grid Size"))
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    for r in rows[1:]:
        if not re.search(pattern, r[cn]) or r[cm] not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        per[r[ci]] = per.get(r[ci], 0.0) + float(r[cv].replace(",", "")) * scale.get(r[cu], 1)
        dims = [int(x) for x in re.findall(r"\d+", r[cg])]
        grid[r[ci]] = dims[0] * dims[1] * dims[2] if len(dims) == 3 else 0
    if largest and per:
        top = max(grid.values())
        per = {i: b for i, b in per.items() if grid[i] == top}
    if not per:
        raise SystemExit(f"no launches of {kernel_regex} with DRAM byte counts in {csv_path}")
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            data = json.load(fh)
    except (OSError, ValueError):
        data = {}
    data[key] = {"dram_bytes_per_launch": group * sum(per.values()) / len(per), "launches": len(per),
                 "launches_per_unit": group, "kernel_regex": kernel_regex, "kernels_sha": kernels_sha()}
    with open(path, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(json.dumps({key: data[key]}))


# ------------------------------------------------------------------ problem
def build_problem(name):
    fac, n, nc, desc = WORKLOADS[name]
    return fac(), n, nc, desc


def host_cpu():
    """(nproc, CPU model) of this host."""
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    import platform
    return os.cpu_count() or 1, model or platform.machine()


def oracle_problem(P, n, nc, gamma):
    """The FP64 CPU oracle on the full workload, its data set (not timed)."""
    import oracle
    O = oracle.Oracle(P.phi_grid(n), nc, gamma=gamma)
    for l in range(O.nlev):
        O.set_bc(l, P.bc_types(O.ghosts(l)["B"]))
    G = O.ghosts(0)
    types = P.bc_types(G["B"])
    O.set_rhs(P.f_grid(n), P.g_values(G["B"], G["nu"], types))
    return O, int((O.types(0) > 0).sum())


def oracle_cycle_seconds(O, threads, cycles):
    """Seconds per oracle cycle (from u = 0, its defects included) with
    `threads` threads; returns (seconds, threads in effect)."""
    import oracle
    used = oracle.set_threads(threads)
    t0 = time.perf_counter()
    O.solve(rtol=0.0, max_cycles=cycles)
    return (time.perf_counter() - t0) / cycles, used


def cycles_reference(name):
    """Cycles to the workload's target of the oracle (written by
    tests/golden/make_bench_cycles.py, which calls only the oracle)."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "bench_cycles.json")) as fh:
            return json.load(fh)[name]["cycles"]
    except (OSError, ValueError, KeyError):
        return None


def cpu_baseline(P, n, nc, gamma, name, cycles_sample, single, fallback_cycles):
    """The oracle as it stands on this host: one cycle of the full workload
    with every host thread (its OpenMP loops) and, if `single`, with one,
    scaled by the oracle's own cycle count to 1e-10."""
    nproc, model = host_cpu()
    O, nunk = oracle_problem(P, n, nc, gamma)
    cyc = cycles_reference(name) or fallback_cycles
    s_all, used = oracle_cycle_seconds(O, nproc, cycles_sample)
    out = {"value": nunk / (s_all * cyc), "unit": "unknowns/s", "cores": used, "kind": "oracle",
           "sample": f"{cycles_sample} oracle cycle(s) of the full {name} problem ({nunk} unknowns) on {used} "
                     f"threads, {s_all:.2f} s per cycle, scaled by the oracle's {cyc} cycles to the target; "
                     f"oracle setup not timed",
           "nproc": nproc, "cpu": model, "s_per_cycle": s_all, "cycles_to_target": cyc}
    if single:
        s_one, _ = oracle_cycle_seconds(O, 1, cycles_sample)
        out["single_core"] = {"value": nunk / (s_one * cyc), "unit": "unknowns/s", "cores": 1,
                              "s_per_cycle": s_one}
    import oracle
    oracle.set_threads(1)
    return out


# ------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, _ = dist()
    if rank != 0:
        return
    P, n, nc, desc = build_problem(args.config)
    cyc = cycles_reference(args.config)
    nproc, model = host_cpu()
    t_total0 = time.perf_counter()
    O, nunk = oracle_problem(P, n, nc, args.gamma)
    per_cycle = []
    used = 1
    for i in range(args.warmup + args.steps):
        sec, used = oracle_cycle_seconds(O, nproc, 1)
        if i >= args.warmup:
            per_cycle.append(sec)
    wall = time.perf_counter() - t_total0
    sec = statistics.mean(per_cycle)
    value = nunk / (sec * cyc) if cyc else None
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.config, "description": desc, "unknowns": nunk,
                       "cycle": "V(2,1)" if args.gamma == 1 else "W(2,1)"},
            "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": used, "kind": "oracle",
                             "nproc": nproc, "cpu": model,
                             "sample": f"one oracle cycle per step on the full {args.config} problem on {used} "
                                       f"threads; unknowns/s = unknowns / (s per cycle x the oracle's {cyc} "
                                       f"cycles to 1e-10); oracle setup not timed"},
            "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batch
def build_batch(count, stream, rtol=1e-10, max_cycles=100):
    """Seeded stars (inputs.star_params) as one gcmg batch with their data set."""
    import torch
    from paper_1111_0983_gb300 import gcmg
    probs = [inputs.star(i) for i in range(count)]
    sizes = [P.meta["n"] for P in probs]
    B = gcmg.Batch([P.phi_grid(n) for P, n in zip(probs, sizes)], 33, stream=stream, rtol=rtol,
                   max_cycles=max_cycles)
    for S, P, n in zip(B.domains, probs, sizes):
        for l in range(S.nlev):
            S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
        G = S.ghosts(0)
        g = P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))
        S.set_rhs(torch.from_numpy(P.f_grid(n)).cuda(), torch.from_numpy(g).cuda())
    unknowns = sum(S.num_unknowns(0) for S in B.domains)
    # fused-sweep bytes of one cycle: 12 B (FP32) per inside node per sweep,
    # nu1 + nu2 sweeps on every level of every domain
    n_in = 0
    for S in B.domains:
        for l in range(S.nlev - 1):
            n_in += int(((S.node_types(l) & 3) == 1).sum())
    return B, sizes, unknowns, 12 * 3 * n_in


def run_batch_measure(B, steps, warmup, stream, flush):
    import torch
    best, tune_ms = B.autotune()
    for _ in range(warmup):
        stats, m = B.solve()
    ms, cyc = 0.0, []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        stats, m = B.solve()
        b.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        cyc.append(m)
    bad = [i for i, st in enumerate(stats) if not st["converged"]]
    return ms / steps, cyc, best, tune_ms, bad, stats


def fmg_entry(name, stream, flush):
    """Time to discretisation accuracy in plain FP64: full multigrid with nu
    cycles a level against V-cycles from u = 0 (device time, CUDA events)."""
    import torch
    from paper_1111_0983_gb300 import gcmg
    P, n, nc, desc = build_problem(name)
    S = gcmg.Solver(P.phi_grid(n), nc, stream=stream, precision=0, rtol=1e-300, max_cycles=1)
    for l in range(S.nlev):
        S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
    rhs = []
    for l in range(S.nlev):
        nl = S.shape(l)[0]
        G = S.ghosts(l)
        g = P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))
        rhs.append((torch.from_numpy(P.f_grid(nl)).cuda(), torch.from_numpy(g).cuda()))
    S.set_rhs(*rhs[0])
    T = S.node_types(0) & 3
    ue = torch.from_numpy(P.u_grid(n)).cuda()
    m = torch.from_numpy(T == 1).cuda()
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")

    def err():
        return float((u - ue).abs()[m].max())

    def timed(fn):
        flush.zero_()
        u.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    # discretisation error: the converged solution's
    S2 = gcmg.Solver(P.phi_grid(n), nc, stream=stream, precision=0, rtol=1e-12, max_cycles=200)
    for l in range(S2.nlev):
        S2.set_bc_types(l, P.bc_types(S2.ghosts(l)["B"]))
    S2.set_rhs(*rhs[0])
    u.zero_()
    S2.solve(u)
    disc = err()
    out = {"workload": name, "description": desc, "precision": "f64", "disc_error": disc, "fmg": [], "vcycles": None}

    def fmg(nu):
        for l in range(1, S.nlev):
            S.set_rhs_level(l, *rhs[l])
        S.fmg(nu, u)

    for nu in (1, 2, 3, 6):
        fmg(nu)   # warm
        ms = timed(lambda: fmg(nu))
        out["fmg"].append({"nu": nu, "ms": ms, "error": err(), "error_over_disc": err() / disc})
    # fewest V-cycles from 0 that reach 1.1 x the discretisation error, timed as one solve
    for k in range(1, 40):
        S3 = gcmg.Solver(P.phi_grid(n), nc, stream=stream, precision=0, rtol=1e-300, max_cycles=k)
        for l in range(S3.nlev):
            S3.set_bc_types(l, P.bc_types(S3.ghosts(l)["B"]))
        S3.set_rhs(*rhs[0])
        u.zero_()   # the solve starts from u
        S3.solve(u)
        if err() <= 1.1 * disc:
            ms = timed(lambda: S3.solve(u))
            out["vcycles"] = {"cycles": k, "ms": ms, "error": err(), "error_over_disc": err() / disc}
            S3.close()
            break
        S3.close()
    S.close()
    S2.close()
    return out


# ----------------------------------------------------------------- gcmg arm
def secondary(name, rtol, precision, args, stream, flush):
    """Time the same form on another workload (plain FP64 and mixed)."""
    import torch
    from paper_1111_0983_gb300 import gcmg
    P, n, nc, desc = build_problem(name)
    out = {"workload": name, "description": desc, "rtol": rtol}
    if name == "flower4097":
        out["note"] = FP64_FLOOR_NOTE
    for prec in (0, 1):
        t0 = time.perf_counter()
        S = gcmg.Solver(P.phi_grid(n), nc, stream=stream, precision=prec, gamma=args.gamma, rtol=rtol,
                        max_cycles=256)
        if P.dim == 3 and SWEEP3D >= 0:
            S.set_sweep3d(SWEEP3D)
        if P.dim == 3 and BOUNDARY3D >= 0:
            S.set_boundary3d(BOUNDARY3D)
        for l in range(S.nlev):
            S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
        G = S.ghosts(0)
        g_h = P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))
        S.set_rhs(torch.from_numpy(P.f_grid(n)).cuda(), torch.from_numpy(g_h).cuda())
        u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
        for _ in range(2):
            u.zero_()
            S.solve(u)
        ms, cyc = 0.0, []
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            u.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = S.solve(u)
            b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
            cyc.append(st["cycles"])
            if not st["converged"]:
                out["f64" if prec == 0 else "mixed"] = {"converged": False, "rel": float(st["rel_residual"])}
                break
        else:
            k = max(1, min(args.steps, 3))
            rec = {"value": S.num_unknowns(0) * k / (ms / 1e3), "unit": "unknowns/s", "ms_per_solve": ms / k,
                   "cycles": cyc}
            # the fine-level fused sweep of this form, timed live with CUDA events
            # around each launch in one instrumented solve
            n_in = int(((S.node_types(0) & 3) == 1).sum())
            flush.zero_()
            u.zero_()
            S.set_kernel_timing(S.KERNEL_SMOOTH)
            S.solve(u)
            kl, kms, kbytes = S.kernel_timing_ex()
            S.set_kernel_timing(-1)
            if kl:
                alg = kbytes / kl if kbytes > 0 else (24 if prec == 0 else 12) * n_in
                gbs = alg / (kms / kl / 1e3) / 1e9
                peak = measured_peaks()[0].get("hbm_gbs")
                kernel = (sweep3d_kernel(prec)[1] if P.dim == 3 else
                          "k_rb_fused2d" if prec == 0 or kbytes <= 0 else
                          "k_relax2d (interior sweep + ghost and band sweeps)")
                rec["fine_sweep"] = {"kernel": kernel, "alg_bytes_per_launch": alg,
                                     "avg_launch_ms": kms / kl, "achieved_GBs": gbs,
                                     "frac_of_measured_hbm": gbs / peak if peak else None}
            out["f64" if prec == 0 else "mixed"] = rec
        out["unknowns"] = S.num_unknowns(0)
        out["setup_s_" + ("f64" if prec == 0 else "mixed")] = time.perf_counter() - t0
        S.close()
    return out


SWEEP3D = -1   # --sweep3d
BOUNDARY3D = -1   # --boundary3d


def sweep3d_kernel(precision):
    """Key and description of the 3D fine-level interior sweep that runs."""
    mode = 3 if SWEEP3D < 0 else SWEEP3D
    if mode == 2 and precision == 0:
        mode = 1   # the row-span kernel is FP32 only
    return {0: ("zmarch", "k_rb_zmarch (fine level: red + black 7-point sweep in one pass, planes staged in "
                          "shared memory)"),
            1: ("stream3d", "k_rb_stream3d (fine level: red + black 7-point sweep in one pass, tiles marching "
                            "along axis 0 with the planes in registers)"),
            2: ("span3d", "k_rb_span3d (fine level: red + black 7-point sweep in one pass, windows covering each "
                          "row's unknowns, planes in registers)"),
            3: ("rows", "k_rb_rows x 2 (fine level: the red then the black half-sweep in place over 64-node "
                        "segments of the rows holding inside nodes; one sweep = two launches, timed together)")}[mode]


def make_solver(P, n, nc, stream, precision, gamma, rtol, **kw):
    import torch
    from paper_1111_0983_gb300 import gcmg
    S = gcmg.Solver(P.phi_grid(n), nc, stream=stream, precision=precision, gamma=gamma, rtol=rtol,
                    max_cycles=256, **kw)
    if P.dim == 3 and SWEEP3D >= 0:
        S.set_sweep3d(SWEEP3D)
    if P.dim == 3 and BOUNDARY3D >= 0:
        S.set_boundary3d(BOUNDARY3D)
    for l in range(S.nlev):
        S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
    G = S.ghosts(0)
    f_h = P.f_grid(n)
    g_h = P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))
    S.set_rhs(torch.from_numpy(f_h).cuda(), torch.from_numpy(g_h).cuda())
    return S, f_h, g_h


def timed_solves(S, u, steps, stream, flush):
    """Device ms of `steps` solves from u = 0 (CUDA events on the stream, L2
    flushed before each) and their cycle counts."""
    import torch
    ms, cyc, st = 0.0, [], None
    for _ in range(steps):
        flush.zero_()
        u.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = S.solve(u)
        b.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        cyc.append(st["cycles"])
        if not st["converged"]:
            raise RuntimeError(f"solve did not converge: {st}")
    return ms / steps, cyc, st


def paper_method_entry(name, stream, flush, steps):
    """The paper's method on a workload (plain FP64, the junction relaxation
    off, V(2,1) and W(2,1) cycles, lambda = 5): device time, cycles and the
    convergence factor beside the oracle's (same algorithm) on the same
    problem, next to the default cycle with the junction solve."""
    import torch
    P, n, nc, desc = build_problem(name)
    out = {"workload": name, "description": desc, "precision": "f64", "forms": []}
    for label, gamma, kw in (("paper V(2,1)", 1, dict(junction_solve=0, junction_sweeps=0)),
                             ("paper W(2,1)", 2, dict(junction_solve=0, junction_sweeps=0)),
                             ("V(2,1) + junction solve", 1, {})):
        S, _, _ = make_solver(P, n, nc, stream, 0, gamma, 1e-10, **kw)
        u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
        S.solve(u)
        try:
            ms, cyc, st = timed_solves(S, u, max(1, min(steps, 2)), stream, flush)
            ok = True
        except RuntimeError:
            u.zero_()
            st, ms, cyc, ok = S.solve(u), None, [S.solve(u)["cycles"]], False
        rel = st["rel"]
        rho = float(np.median(rel[2:] / rel[1:-1])) if len(rel) > 3 else None
        rec = {"form": label, "converged": ok, "cycles": cyc[-1], "ms_per_solve": ms,
               "unknowns_per_s": S.num_unknowns(0) / (ms / 1e3) if ms else None, "rho_median": rho,
               "diverged": bool(st.get("diverged", False))}
        out["unknowns"] = S.num_unknowns(0)
        S.close()
        # the oracle's factor on the same problem and cycle (paper-mode forms only)
        if kw:
            import oracle
            O = oracle.Oracle(P.phi_grid(n), nc, gamma=gamma, junction_solve=0, junction_sweeps=0)
            for l in range(O.nlev):
                O.set_bc(l, P.bc_types(O.ghosts(l)["B"]))
            G = O.ghosts(0)
            O.set_rhs(P.f_grid(n), P.g_values(G["B"], G["nu"], P.bc_types(G["B"])))
            oracle.set_threads(os.cpu_count() or 1)
            _, norms, _ = O.solve(rtol=1e-10, max_cycles=min(len(rel) - 1, 12))
            oracle.set_threads(1)
            r = norms[2:] / norms[1:-1]
            rec["oracle_rho_median"] = float(np.median(r)) if len(r) else None
        out["forms"].append(rec)
    return out


def run_gcmg(args):
    import torch
    import torch.distributed as tdist

    from paper_1111_0983_gb300 import gcmg

    rank, world, local = dist()
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()

    P, n, nc, desc = build_problem(args.config)
    precision = 1 if args.precision == "mixed" else 0
    t_setup = time.perf_counter()
    S, f_h, g_h = make_solver(P, n, nc, stream, precision, args.gamma, args.rtol)
    setup_s = time.perf_counter() - t_setup
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
    nunk = S.num_unknowns(0)
    n_in = int(((S.node_types(0) & 3) == 1).sum())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        u.zero_()
        S.solve(u)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = gcmg.launch_counter()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    cycles = []
    t_wall0 = time.perf_counter()
    st = None
    for k in range(args.steps):
        flush.zero_()
        u.zero_()
        ev[k][0].record(stream)
        st = S.solve(u)
        ev[k][1].record(stream)
        cycles.append(st["cycles"])
        if not st["converged"]:
            raise RuntimeError(f"solve did not converge: {st}")
    barrier()
    wall = time.perf_counter() - t_wall0
    launches = gcmg.launch_counter() - launches0
    clk = clocks.stop()
    rel_hist = st["rel"]
    # further passes of the same solves with CUDA events around every
    # fine-level launch of the interior sweep (and, in 2D, of every
    # boundary-block launch): events cannot live inside the graph's loop body
    S.set_kernel_timing(S.KERNEL_SMOOTH)
    for k in range(args.steps):
        flush.zero_()
        u.zero_()
        S.solve(u)
    k_launches, k_ms, k_bytes = S.kernel_timing_ex()
    b_launches, b_ms, b_bytes = 0, 0.0, 0.0
    if P.dim == 2:
        S.set_kernel_timing(S.KERNEL_BOUNDARY)
        for k in range(args.steps):
            flush.zero_()
            u.zero_()
            S.solve(u)
        b_launches, b_ms, b_bytes = S.kernel_timing_ex()
    if args.profile_solve:
        # plain launches (kernel timing keeps the graph off) inside the profiler range
        S.set_kernel_timing(S.KERNEL_DEFECT)
        u.zero_()
        S.solve(u)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        u.zero_()
        S.solve(u)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    S.set_kernel_timing(-1)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t.item())
    value = nunk * args.steps * world / (ms / 1e3)

    # end to end through the host-buffer entry point
    f_pin = torch.from_numpy(f_h).pin_memory().numpy()
    g_pin = torch.from_numpy(g_h).pin_memory().numpy()
    u_pin = torch.empty(S.shape(0), dtype=torch.float64).pin_memory().numpy()
    S.solve_host(f_pin, g_pin, u_pin)
    barrier()
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.solve_host(f_pin, g_pin, u_pin)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_t)
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = nunk * args.steps * world / e2e_s

    peaks, peak_kind = measured_peaks()
    peak = peaks.get("hbm_gbs")
    # the interior sweep: both colours in one launch (2D strips / tiles, 3D
    # z-march) reading u and f and writing u once per inside node, plus in
    # the merged FP32 2D relaxation the boundary blocks' values (the library
    # gives those bytes)
    elt = 4 if precision else 8
    alg_bytes = k_bytes / k_launches if k_launches and k_bytes > 0 else 3 * elt * n_in
    avg_ms = k_ms / max(k_launches, 1)
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9 if k_launches else None
    merged = P.dim == 2 and precision == 1 and b_launches > 0
    kern = ("relax2d" if merged else "fused2d") if P.dim == 2 else sweep3d_kernel(precision)[0]
    kname = f"rb_{kern}_{'f64' if precision == 0 else 'f32'}_{args.config}"
    kdesc = {"relax2d": "k_relax2d (fine level: interior sweep + ghost and band sweeps in one launch)",
             "fused2d": "k_rb_fused2d (fine level, red + black sweep)"}.get(kern) or sweep3d_kernel(precision)[1]
    sweep = {"bound": "hbm", "kernel": kdesc, "achieved": achieved,
             "peak": peak, "peak_kind": f"{peak_kind} hbm_gbs", "unit": "GB/s",
             "frac": (achieved / peak) if achieved and peak else None, "traffic": traffic_for(kname),
             "alg_bytes_per_launch": alg_bytes, "alg_bytes_note": f"{3 * elt} B x {n_in} inside nodes"
             if P.dim == 3 else None, "avg_launch_ms": avg_ms, "launches_timed": k_launches,
             "share_of_solve": (k_ms / ms) if ms > 0 else None}
    if P.dim == 3 and kern == "rows":
        sweep["launch_note"] = ("a unit is one sweep: the red and the black launch, timed together; the kernels "
                                "that take most of the solve's time are the boundary phases' short list launches "
                                "(latency bound), see the launch list under profiles/")
    roofline = sweep
    if b_launches:
        bname = f"{'relax2d' if merged else 'local_bz'}_{'f64' if precision == 0 else 'f32'}_{args.config}"
        b_ach = (b_bytes / b_launches) / (b_ms / b_launches / 1e3) / 1e9 if b_ms > 0 else None
        bdesc = ("k_relax2d (one FP32 relaxation: interior strips and boundary blocks in one launch, every level)"
                 if merged else "k_local (2D boundary blocks: ghost sweep + lambda band sweeps in shared memory, "
                 "every level)")
        roofline = {"bound": "hbm", "kernel": bdesc, "achieved": b_ach, "peak": peak,
                    "peak_kind": f"{peak_kind} hbm_gbs", "unit": "GB/s",
                    "frac": (b_ach / peak) if b_ach and peak else None, "traffic": traffic_for(bname),
                    "alg_bytes_per_launch": b_bytes / b_launches, "avg_launch_ms": b_ms / b_launches,
                    "launches_timed": b_launches}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 cycles + f64 refinement" if precision else "f64", "data": "synthetic",
                "config": {"workload": args.config, "description": desc, "unknowns": nunk, "inside": n_in,
                           "ghosts": S.num_ghosts(0), "levels": S.nlev, "n_coarse": nc,
                           "cycle": "V(2,1)" if args.gamma == 1 else "W(2,1)", "lambda": 5, "rtol": args.rtol,
                           "cycles_per_solve": cycles, "l2": "flushed between steps (256 MB write)",
                           "parallelism": f"replicas x{world}", "setup_s": setup_s},
                "rho": [float(x) for x in (rel_hist[1:] / rel_hist[:-1])],
                "roofline": roofline, "sweep_roofline": sweep, "clocks": clk, "gpu_launches": launches,
                "e2e": {"value": e2e_value, "unit": "unknowns/s",
                        # f is page-locked: the device reads it at the inside nodes only
                        "h2d_bytes_per_step": int(8 * n_in + g_h.nbytes),
                        "d2h_bytes_per_step": int(u_pin.nbytes),
                        "note": "gcmg_solve_host with page-locked buffers: the device reads f at the "
                                "inside nodes from host memory, g is copied, the device stores u (n^d) "
                                "into host memory"},
                "wall_s": wall}
        S.close()
        del S
        if precision == 1 and world == 1 and args.fp64:
            # the plain FP64 GPU solve of the same workload (the metric's comparison)
            t0 = time.perf_counter()
            rt64 = max(args.rtol, FP64_FLOOR_RTOL.get(args.config, args.rtol))
            S64, _, _ = make_solver(P, n, nc, stream, 0, args.gamma, rt64)
            setup64 = time.perf_counter() - t0
            u.zero_()
            S64.solve(u)
            ms64, cyc64, st64 = timed_solves(S64, u, max(1, min(args.steps, 3)), stream, flush)
            line["fp64"] = {"value": nunk / (ms64 / 1e3), "unit": "unknowns/s", "ms_per_solve": ms64,
                            "cycles": cyc64, "rtol": rt64, "rel_residual": st64["rel_residual"],
                            "setup_s": setup64}
            if rt64 > args.rtol:
                line["fp64"]["note"] = (f"plain FP64 cannot reach {args.rtol:g} on this grid (the rounding of u in "
                                        f"its smoother keeps the defect near {rt64:g} of ||(f, g)||); timed to "
                                        f"{rt64:g}, so the speed-up understates the mixed form's")
            line["speedup_vs_fp64"] = (ms64 * args.steps) / ms
            S64.close()
            del S64
        if args.also and world == 1:
            line["also"] = []
            for item in args.also.split(","):
                name, rt = item.split(":")
                if name == args.config:
                    continue
                line["also"].append(secondary(name, float(rt), precision, args, stream, flush))
        if args.paper and world == 1:
            line["paper_method"] = paper_method_entry(args.paper, stream, flush, args.steps)
        if args.batch and world == 1:
            t0 = time.perf_counter()
            B, sizes, bun, fused_bytes = build_batch(args.batch, stream)
            bsetup_s = time.perf_counter() - t0
            profile_batch = args.batch_profile
            bms, bcyc, best, tune_ms, bad, bst = run_batch_measure(B, max(1, min(args.steps, 3)), 2, stream, flush)
            line["batch"] = {"workload": f"stars{args.batch}", "domains": args.batch,
                             "grid_sizes": {str(k): sizes.count(k) for k in sorted(set(sizes))},
                             "unknowns": bun, "value": bun / (bms / 1e3), "unit": "unknowns/s",
                             "ms_per_solve": bms, "refinement_steps": bcyc, "setup_s": bsetup_s,
                             "cycles_max": max(x["cycles"] for x in bst),
                             "cycles_median": statistics.median(x["cycles"] for x in bst),
                             "tile_variant": ["strips of 8 rows", "strips of 16 rows", "strips of 32 rows"][best],
                             "autotune_ms_fused_sweeps_per_cycle": tune_ms,
                             "fused_sweep_GBs": fused_bytes / (min(tune_ms) / 1e3) / 1e9,
                             "converged": len(bad) == 0, "not_converged": bad,
                             "worst_rel": max(x["rel_residual"] for x in bst)}
            if profile_batch:
                B.set_graph(False)
                B.solve()   # warm the plain-launch form
                torch.cuda.synchronize()
                torch.cuda.profiler.start()
                B.solve()
                torch.cuda.synchronize()
                torch.cuda.profiler.stop()
                B.set_graph(True)
            B.close()
        if args.fmg and world == 1:
            line["fmg"] = fmg_entry(args.fmg, stream, flush)
        if args.learned and world == 1:
            from paper_1111_0983_gb300 import learn
            t0 = time.perf_counter()
            cmp = learn.compare_forms(learn.load_weights(), [learn.TEST_BASE + i for i in range(args.learned)])
            cmp["workload"] = f"learned guess, {args.learned} held-out stars at 513^2, Gaussian f, g = 0"
            cmp["wall_s"] = time.perf_counter() - t0
            line["learned"] = cmp
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(P, n, nc, args.gamma, args.config, args.cpu_sample_cycles,
                                                bool(args.cpu_single), statistics.median(cycles))
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.barrier()
        tdist.destroy_process_group()


def main():
    global SWEEP3D, BOUNDARY3D
    args = parse()
    SWEEP3D, BOUNDARY3D = args.sweep3d, args.boundary3d
    if args.write_traffic:
        write_traffic(*args.write_traffic, group=args.traffic_group)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gcmg(args)


if __name__ == "__main__":
    main()
