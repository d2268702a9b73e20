#!/usr/bin/env python
"""Benchmark of the lumped pressure-Helmholtz multigrid solve on GB300.

One step = one complete solve H^ x = b (PCG preconditioned by one V-cycle per
iteration, x0 = 0, stopped at ||r||/||b|| < 1e-8) on the paper-scale shell:
icosahedral refinement 6 (81,920 columns) x 64 layers, 5 levels, FP64
(Table "Grid setup", LO).  The right-hand side is seeded N(0,1) per cell, on
the device before the timed region.  Alongside the FP64 solves/s the line
reports the mixed form (FP32 V-cycle, FP64 Krylov and coarsest level), the
V-cycle bandwidth of both forms against the measured HBM peak, the roofline
of the dominant kernel (timed live with CUDA events inside the timed region),
an end-to-end number through host buffers, the clocks seen and the CPU oracle
timed on a bounded sample.

--impl reference times the CPU oracle itself on the same workload (one PCG
iteration per step, scaled to solves/s by the iteration count of the full
solve).  Under torchrun every rank solves its own copy of the problem
(replicas: the solve is not sharded across GPUs), rank 0 prints.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "V-cycle HBM GB/s (% of peak); solves/s at 81920x64, FP64 vs mixed @1e-8"
UNIT = "solves/s"
WORKLOAD = "r6x64"


def workload_desc(name):
    import hmg_inputs as gi
    w = gi.WORKLOADS[name]
    shell = (f"icosahedral refinement {w['refinement']} ({gi.ncolumns(w['refinement'])} columns) x "
             f"{w['nlayers']} layers, R = 6371 km, H = 10 km, ")
    if w.get("order") == "nlo":
        return shell + (f"next-to-lowest order (DG1 pressure, 6 unknowns per cell), the NLO level plus "
                        f"{w['nlevels']} lowest-order levels, nu_CFL = 8, omega = 0.8, 2 pre / 2 post sweeps, "
                        "2 coarsest sweeps, GMRES(30) to 1e-5")
    return shell + (f"{w['nlevels']} levels, nu_CFL = 8, omega = 0.8, "
                    "2 pre / 2 post sweeps, 2 coarsest sweeps, PCG to 1e-8")
def bench_config(name):
    """The config dict of the JSON line (the same for both arms)."""
    import hmg_inputs as gi
    w = gi.WORKLOADS[name]
    return {"workload": f"{name}: {workload_desc(name)}", "ncols": gi.ncolumns(w["refinement"]),
            "nlayers": w["nlayers"], "ncells": gi.ncells(w["refinement"], w["nlayers"]), "nlevels": w["nlevels"],
            "rhs": "N(0,1) per cell, seed 0", "krylov": "CG",
            "l2": "working set > 1 GB, larger than the 126 MB L2: no flush"}


# Peak host memory of one oracle sample process at r6x64 (measured 2.7 GB).
ORACLE_SAMPLE_GB = 3.0

# PCG iterations of the full FP64 solve of this workload (oracle and GPU agree;
# asserted by tests/test_gpu_fullsize.py).  Used to scale the oracle sample.
ORACLE_ITERATIONS = 11

# Derived FP64 peak of GB300: 152 SMs x 4 sub-partitions, each retiring one
# 32-lane FP64 FMA warp instruction per 64 cycles (measured: issue interval
# and dependent latency both 64 cycles), 2 flops per FMA, 2070 MHz maximum SM
# clock: 152 * 4 * 32 / 64 * 2 * 2.07e9 = 1.259 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 4 * 32 / 64 * 2 * 2.07e9 / 1e12
FALLBACK_HBM_GBS = 6800.0
REFERENCE_BUDGET_S = 150.0   # wall time of the --impl reference timed + warm-up steps
# DRAM bytes per launch of the dominant kernel class of the r6x64 bench (FP64
# half-column sweeps on the finest level: two plain sweeps and one with the
# fused r.z per V-cycle), from an ncu capture of dram__bytes_read.sum +
# dram__bytes_write.sum of this bench command: 292.8 MB (plain, three
# launches), 327.8 MB (with the dot)
TRAFFIC_SWEEP_L0_R6X64 = 304.5e6


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------- byte / flop models
# Algorithmic bytes per fine cell of each kernel (stored coefficients and
# vectors once per kernel; neighbour re-reads of u are not counted), s = bytes
# per scalar of the level's type, nz = layers; per-column data (3 neighbour
# indices + pad = 16 B, 3 couplings + sum = 4 s) is spread over nz cells.

def kernel_bytes_per_cell(kernel, s, nz, s_b=None, s_out=None, s_c=None, fused_prolong=False):
    s_b = s_b or s
    s_out = s_out or s
    s_c = s_c or s
    col = (16 + 4 * s) / nz
    if kernel == "sweep0":
        extra = 4 if (s == 4 and s_b == 8) else 0          # FP32 copy of an FP64 b
        return s_b + 2 * s + s_out + extra
    if kernel == "sweep":
        return 4 * s + s_out + col + (s_c / 4 if fused_prolong else 0)
    if kernel == "resid_restrict":
        return 4 * s + s_c / 4 + col
    if kernel == "prolong":
        return 2 * s + s_c / 4
    if kernel == "apply":
        return 4 * s + col
    raise ValueError(kernel)


# FP64 operations per cell (FMA counted as 2 flops, MUL/ADD as 1)
KERNEL_FLOPS = {"sweep0": 5, "sweep": 13, "resid_restrict": 12.5, "prolong": 1, "apply": 11}


def useful_bandwidth(breakdown, levels_ncells, nz, hbm_gbs):
    """Per kernel class and level of an FP64 solve, the paper's "useful
    bandwidth" (Sec. 5.4, performance model): model bytes of all launches over
    their traced time, with the FP64 rate beside it (the GB300 bound of these
    kernels).  breakdown: {(kernel, level): (launches, ms)}."""
    out = {}
    for (k, lev), (n, ms) in sorted(breakdown.items(), key=lambda kv: (kv[0][1], kv[0][0])):
        if k not in KERNEL_FLOPS or ms <= 0:
            continue
        cells = levels_ncells[lev]
        gbs = kernel_bytes_per_cell(k, 8, nz) * cells * n / (ms * 1e-3) / 1e9
        tfl = KERNEL_FLOPS[k] * cells * n / (ms * 1e-3) / 1e12
        out[f"{k}@{lev}"] = {"launches": n, "us_per_launch": round(1e3 * ms / n, 2), "GB_s": round(gbs, 1),
                             "frac_hbm": round(gbs / hbm_gbs, 4), "TFLOP_s": round(tfl, 4),
                             "frac_fp64": round(tfl / FP64_PEAK_TFLOPS, 4)}
    return out


def vcycle_bytes(levels_ncells, nz, mixed, nu_pre=2, nu_post=2, n_coarse=2):
    """Model bytes of one V-cycle (sum of its kernels)."""
    total = 0.0
    L = len(levels_ncells)
    for lev, n in enumerate(levels_ncells):
        fp32 = mixed and lev < L - 1
        s = 4 if fp32 else 8
        s_c = (4 if (mixed and lev + 1 < L - 1) else 8) if lev < L - 1 else s
        s_b = 8 if lev == 0 else s
        out0 = 8 if lev == 0 else s
        if lev == L - 1:
            total += n * kernel_bytes_per_cell("sweep0", s, nz, s_b=s_b)
            total += (n_coarse - 1) * n * kernel_bytes_per_cell("sweep", s, nz)
            continue
        sb_after = s  # later kernels read the level's own copy of b
        total += n * kernel_bytes_per_cell("sweep0", s, nz, s_b=s_b)
        total += (nu_pre - 1) * n * kernel_bytes_per_cell("sweep", sb_after, nz)
        total += n * kernel_bytes_per_cell("resid_restrict", s, nz, s_c=s_c)
        if not fp32:
            total += n * kernel_bytes_per_cell("prolong", s, nz, s_c=s_c)
        for i in range(nu_post):
            last = i == nu_post - 1
            total += n * kernel_bytes_per_cell("sweep", s, nz, s_out=out0 if last else s, s_c=s_c,
                                               fused_prolong=(fp32 and i == 0))
    return total


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (every 100 ms) during the timed region."""

    QUERY = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def mark(self, start):
        if start:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def summary(self):
        import datetime
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def stamp(x):
            try:
                return datetime.datetime.strptime(x, "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                return None

        t0, t1 = getattr(self, "t0", None), getattr(self, "t1", None)
        inside = [r for r in rows if t0 and t1 and stamp(r[0]) is not None and t0 - 0.05 <= stamp(r[0]) <= t1 + 0.05]
        window = "timed region" if inside else "whole run (no sample inside the timed region)"
        rows = inside or rows

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "window": window,
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ---------------------------------------------------------------- distributed

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, world, device):
    """Max of a float over all ranks (identity for one rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- CPU oracle

def oracle_sample(workload, pcg_iterations, threads_note=True):
    """Time the oracle's first `pcg_iterations` PCG iterations (setup excluded)."""
    import numpy as np  # noqa: F401
    import hmg_inputs as gi
    from oracle import helmholtz, krylov, mesh, multigrid
    w = gi.WORKLOADS[workload]
    t0 = time.perf_counter()
    ms = mesh.hierarchy(w["refinement"], w["nlevels"])
    prm = helmholtz.Params(refinement=w["refinement"], nlayers=w["nlayers"])
    ops = helmholtz.assemble_hierarchy(ms, prm)
    setup_s = time.perf_counter() - t0
    b = gi.rhs(ops[0].ncells)
    t0 = time.perf_counter()
    krylov.pcg(ops[0].H.dot, lambda v: multigrid.vcycle(ops, v), b, rtol=1e-8, max_iter=pcg_iterations)
    return time.perf_counter() - t0, setup_s


def cpu_baseline_subprocess(workload, iterations, copies=None):
    """The oracle on the host's cores: `copies` (default: every core the
    process may use) independent single-threaded processes, each timing the
    same bounded sample of the solve, started together.  solves/s is the sum
    over the copies (independent problems, as the GPU arm's replicas), and
    the single-copy figure is reported beside it."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    if copies is None:
        try:
            copies = len(os.sched_getaffinity(0))
        except AttributeError:
            copies = os.cpu_count() or 1
    # at most half the available host memory (one r6x64 sample peaks at 2.7 GB)
    try:
        with open("/proc/meminfo") as f:
            avail_gb = next(int(l.split()[1]) for l in f if l.startswith("MemAvailable")) / 1e6
        copies = min(copies, max(1, int(0.5 * avail_gb / ORACLE_SAMPLE_GB)))
    except (OSError, StopIteration, ValueError):
        copies = 1
    copies = max(1, int(copies))
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", workload, "--oracle-iterations",
           str(iterations)]
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
             for _ in range(copies)]
    solve_s = []
    err = None
    for p in procs:
        try:
            out, e = p.communicate(timeout=900)
        except subprocess.TimeoutExpired:
            p.kill()
            out, e = p.communicate()
        if p.returncode != 0:
            err = (e or "")[-400:]
            continue
        d = json.loads(out.strip().splitlines()[-1])
        # pcg(max_iter=k) runs k + 1 V-cycles and k operator applications; the
        # full solve runs ORACLE_ITERATIONS + 1 V-cycles.
        solve_s.append((d["seconds"] * (ORACLE_ITERATIONS + 1) / (iterations + 1), d))
    if not solve_s:
        return {"value": None, "unit": UNIT, "cores": copies, "kind": "oracle", "error": err}
    total = sum(1.0 / t for t, _ in solve_s)
    ts = sorted(t for t, _ in solve_s)
    d0 = solve_s[0][1]
    return {"value": total, "unit": UNIT, "cores": len(solve_s), "kind": "oracle",
            "sample": (f"{len(solve_s)} single-threaded copies of the NumPy/SciPy oracle, one per host core, run "
                       f"together; each times the first {iterations} of {ORACLE_ITERATIONS} PCG iterations of the "
                       f"{workload} FP64 solve (setup excluded; copy 0: {d0['seconds']:.1f} s, setup "
                       f"{d0['setup_s']:.1f} s), scaled by {ORACLE_ITERATIONS + 1}/{iterations + 1} V-cycles to one "
                       "solve; value = sum of the copies' solves/s"),
            "seconds_per_solve_median_copy": statistics.median(ts),
            "seconds_per_solve_min_max": [ts[0], ts[-1]]}


# ---------------------------------------------------------------- GPU arm

# NLO column-block sweep, per cell: three 6 x 6 blocks of coefficients (L_l,
# omega Dt_l^-1, L_(l+1)^T), b, u, u' and the forward results written and read
# back (6 unknowns each); the three neighbour blocks (each a 3 x 3 horizontal
# factor times the fixed 2 x 2 vertical one: 66 FMA), the forward and backward
# block products (36 + 72 FMA) and the relaxation (6 FMA): 180 FMA.
NLO_SWEEP_BYTES_PER_CELL = 3 * 36 * 8 + 5 * 6 * 8
NLO_SWEEP_FLOPS_PER_CELL = 2 * (66 + 36 + 72 + 6)
NLO_SWEEP_BYTES_PER_CELL_FP32 = 3 * 36 * 4 + 5 * 6 * 4
# DRAM bytes per launch of the general NLO sweep at r4x64 (ncu capture of
# dram__bytes_read.sum + dram__bytes_write.sum, experiments --only nlo --quick):
# 176.5 + 11.8 MB for the staged FP32 sweep.  The FP64 sweep's capture
# (358.4 + 30.3 MB) predates a restructuring of its load loop, so its traffic
# is reported as unknown.
TRAFFIC_NLO_SWEEP_R4X64 = None
TRAFFIC_NLO_SWEEP_FP32_R4X64 = 188.4e6


def nlo_section(args, world, dev, stream, hbm):
    import torch

    import hmg_inputs as gi
    import paper_1605_00492_gb300 as hmg
    w = gi.WORKLOADS["r4x64nlo"]
    h = hmg.Hierarchy(w["refinement"], w["nlayers"], w["nlevels"])
    h.assemble()
    n = h.nlo_size()
    ncells = n // 6
    b = torch.tensor(gi.nlo_rhs(n), dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": "r4x64nlo: " + workload_desc("r4x64nlo"), "unknowns_pressure": n, "rtol": 1e-5,
           "krylov": "GMRES(30), one NLO V-cycle (column block relaxation, p-coarsening DG1 -> DG0, "
                     "4 lowest-order levels)"}
    for form in ("fp64", "mixed"):
        kw = dict(precision=form, rtol=1e-5, restart=30, max_iter=300)
        for _ in range(2):
            h.nlo_solve(b, out=x, **kw)
        reps = max(5, min(args.steps, 20))
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            _, info = h.nlo_solve(b, out=x, **kw)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev) / reps
        out[form] = {"solves_per_s": round(world / (ms / 1e3), 3), "ms_per_solve": round(ms, 4),
                     "iterations": info["iterations"], "true_rel_residual": info["true_rel_residual"]}
    # the NLO sweep, traced inside FP64 solves
    h.profile_start(kernels=["nlo_sweep"], levels=[0])
    for _ in range(3):
        h.nlo_solve(b, out=x, precision="fp64", rtol=1e-5, restart=30, max_iter=300)
    rec = h.profile_stop()
    cnt, tot = rec.get(("nlo_sweep", 0), (0, 0.0))
    avg_ms = tot / max(cnt, 1)
    tflops = NLO_SWEEP_FLOPS_PER_CELL * ncells / (avg_ms * 1e-3) / 1e12
    gbs = NLO_SWEEP_BYTES_PER_CELL * ncells / (avg_ms * 1e-3) / 1e9
    # the FP32 sweep of the mixed form, bound by memory
    h.profile_start(kernels=["nlo_sweep"], levels=[0])
    for _ in range(3):
        h.nlo_solve(b, out=x, precision="mixed", rtol=1e-5, restart=30, max_iter=300)
    rec32 = h.profile_stop()
    c32, t32 = rec32.get(("nlo_sweep", 0), (0, 0.0))
    ms32 = t32 / max(c32, 1)
    gbs32 = NLO_SWEEP_BYTES_PER_CELL_FP32 * ncells / (ms32 * 1e-3) / 1e9
    out["sweep_roofline_fp32"] = {"bound": "hbm", "achieved": round(gbs32, 1), "peak": hbm, "unit": "GB/s",
                                  "frac": round(gbs32 / hbm, 4), "launches": c32, "avg_us": round(ms32 * 1e3, 2),
                                  "bytes_per_launch": NLO_SWEEP_BYTES_PER_CELL_FP32 * ncells,
                                  "kernel": "nlo_sweep FP32 (mixed form, operands staged through shared memory)",
                                  "traffic": TRAFFIC_NLO_SWEEP_FP32_R4X64}
    out["sweep_roofline"] = {"bound": "alu", "achieved": round(tflops, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                             "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                             "hbm_achieved_GB_s": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4),
                             "kernel": "nlo_sweep (general sweep, 3 of the 4 per V-cycle)",
                             "launches": cnt, "avg_us": round(avg_ms * 1e3, 2),
                             "bytes_per_launch": NLO_SWEEP_BYTES_PER_CELL * ncells,
                             "flops_per_launch": NLO_SWEEP_FLOPS_PER_CELL * ncells,
                             "traffic": TRAFFIC_NLO_SWEEP_R4X64}
    # the velocity-pressure system at NLO (Table "SingleNodePerformance", NLO
    # row: 7.9 million unknowns, GMRES to 1e-5), right-hand side (M2~ R_U, M3 R_P)
    sizes = h.nlo_mixed_sizes()
    ntot = sum(sizes)
    nu = ntot - sizes[3]
    R = torch.tensor(gi.mixed_rhs(nu, sizes[3]), dtype=torch.float64, device=dev)
    Ru, Rp = R.clone(), R.clone()
    Ru[nu:] = 0
    Rp[:nu] = 0
    bvp = torch.cat([h.nlo_mixed_apply(Ru)[:nu], h.nlo_mixed_apply(Rp)[nu:]])
    vp = {"unknowns": int(ntot), "rtol": 1e-5,
          "krylov": "GMRES(30), Schur-complement preconditioner, one NLO V-cycle for H^^-1"}
    for form in ("fp64", "mixed"):
        kw = dict(precision=form, rtol=1e-5, restart=30, max_iter=300)
        h.nlo_mixed_solve(bvp, **kw)
        reps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            _, info = h.nlo_mixed_solve(bvp, **kw)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev) / reps
        vp[form] = {"solves_per_s": round(world / (ms / 1e3), 3), "ms_per_solve": round(ms, 4),
                    "iterations": info["iterations"], "true_rel_residual": info["true_rel_residual"]}
    out["velocity_pressure"] = vp
    h.close()
    return out


def velocity_pressure_section(h, args, world, dev, stream, ev0, ev1):
    """The lowest-order velocity-pressure system (Sec. 4.1): GMRES(30) with the
    Schur-complement preconditioner (Sec. 4.2), to the paper's 1e-5, right-hand
    side (M2~ R_U, M3 R_P)."""
    import torch

    import hmg_inputs as gi
    nhf, nvf, ncl = h.mixed_sizes()
    R = torch.tensor(gi.mixed_rhs(nhf + nvf, ncl), dtype=torch.float64, device=dev)
    ru, rp = R[:nhf + nvf].contiguous(), R[nhf + nvf:].contiguous()
    bu, _ = h.mixed_apply(ru, torch.zeros_like(rp))
    _, bp = h.mixed_apply(torch.zeros_like(ru), rp)
    vp = {"rtol": 1e-5, "krylov": "GMRES(30), Schur-complement preconditioner, one V-cycle for H^^-1",
          "unknowns": int(nhf + nvf + ncl)}
    for form in ("fp64", "mixed"):
        kwvp = dict(precision=form, rtol=1e-5, restart=30, max_iter=300)
        for _ in range(2):
            h.mixed_solve(bu, bp, **kwvp)
        reps = max(5, min(args.steps, 20))
        res = {}

        def step():
            res["info"] = h.mixed_solve(bu, bp, **kwvp)[2]
        tot, per = timed_steps(step, reps, stream)
        ms = max_over_ranks(tot, world, dev) / reps
        infovp = res["info"]
        vp[form] = {"solves_per_s": round(world / (ms / 1e3), 3), "ms_per_solve": round(ms, 4),
                    "ms_per_solve_stats": step_stats(per),
                    "iterations": infovp["iterations"], "true_rel_residual": infovp["true_rel_residual"]}
    return vp


def timed_steps(fn, steps, stream):
    """Run fn() `steps` times between CUDA events recorded on `stream` (one
    event before each step and one after the last, no synchronisation in
    between).  Returns (total ms, [ms of each step])."""
    import torch
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(steps):
        fn()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
    return evs[0].elapsed_time(evs[-1]), per


def step_stats(per):
    return {"min": round(min(per), 4), "median": round(statistics.median(per), 4), "max": round(max(per), 4)}


def small_config_section(args, dev, stream):
    """The r3x16 workload (20,480 cells, 3 levels): L2-resident and bound by
    launch latency, reported as latency per FP64 solve."""
    import torch

    import hmg_inputs as gi
    import paper_1605_00492_gb300 as hmg
    w = gi.WORKLOADS["r3x16"]
    h = hmg.Hierarchy(w["refinement"], w["nlayers"], w["nlevels"])
    h.assemble()
    b = torch.tensor(gi.rhs(h.ncells), dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    kw = dict(precision="fp64", krylov="cg", rtol=1e-8, max_iter=200)
    for _ in range(5):
        _, info = h.solve(b, out=x, **kw)
    reps = max(20, args.steps)
    total, per = timed_steps(lambda: h.solve(b, out=x, **kw), reps, stream)
    h.close()
    return {"workload": "r3x16: " + workload_desc("r3x16"), "ncells": int(b.numel()),
            "latency_ms": step_stats(per), "solves_per_s": round(reps / (total / 1e3), 2),
            "iterations": info["iterations"], "true_rel_residual": info["true_rel_residual"],
            "note": "L2-resident and launch-latency bound: not counted against HBM"}


def adjoint_section(args, dev, stream):
    """Forward + backward of the differentiable solve p = H^(theta)^-1 b at
    r5x64 (1,310,720 cells, 5 levels): loss 1/2 |p - p_t|^2, gradients with
    respect to b and theta (assembly from theta, forward CG solve, re-assembly,
    adjoint CG solve, face contraction), FP64, CG to 1e-8 both ways."""
    import torch

    import hmg_inputs as gi
    import paper_1605_00492_gb300 as hmg
    from paper_1605_00492_gb300.autograd import HelmholtzSolve
    w = gi.WORKLOADS["r5x64a"]
    t0 = time.perf_counter()
    h = hmg.Hierarchy(w["refinement"], w["nlayers"], w["nlevels"])
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    n = h.ncells
    b0 = torch.tensor(gi.rhs(n), dtype=torch.float64, device=dev)
    th0 = torch.tensor(gi.theta(n), dtype=torch.float64, device=dev)
    pt = torch.tensor(gi.ptarget(n), dtype=torch.float64, device=dev)
    kw = dict(precision="fp64", krylov="cg", rtol=1e-8, max_iter=200)

    def step():
        b = b0.clone().requires_grad_(True)
        th = th0.clone().requires_grad_(True)
        p = HelmholtzSolve.apply(h, b, th, kw)
        loss = 0.5 * torch.sum((p - pt) ** 2)
        loss.backward()
        return b.grad, th.grad

    for _ in range(3):
        step()
    reps = max(5, min(args.steps, 20))
    total, per = timed_steps(step, reps, stream)
    # forward alone, same protocol
    def fwd():
        with torch.no_grad():
            HelmholtzSolve.apply(h, b0, th0, kw)
    totf, _ = timed_steps(fwd, reps, stream)
    h.close()
    return {"workload": "r5x64a: " + workload_desc("r5x64a") + ", theta = exp(0.3 N(0,1)) per cell",
            "ncells": n, "fwd_bwd_ms": step_stats(per), "fwd_bwd_per_s": round(reps / (total / 1e3), 3),
            "fwd_ms": round(totf / reps, 4), "build_s": round(t_build, 3),
            "what": "assemble(theta) + CG solve; backward: assemble(theta) + adjoint CG solve + theta face "
                    "contraction; loss 1/2|p - p_t|^2"}


def large_config_section(args, dev, stream, hbm):
    """The r7x128 workload (327,680 columns x 128 layers = 41.9 M cells, 6
    levels), both forms: solves/s and the V-cycle's model bytes over time."""
    import torch

    import hmg_inputs as gi
    import paper_1605_00492_gb300 as hmg
    w = gi.WORKLOADS["r7x128"]
    t0 = time.perf_counter()
    h = hmg.Hierarchy(w["refinement"], w["nlayers"], w["nlevels"])
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    h.assemble()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    n = h.ncells
    b = torch.tensor(gi.rhs(n), dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    out = {"workload": "r7x128: " + workload_desc("r7x128"), "ncells": n,
           "setup_s": {"build_hierarchy": round(t1 - t0, 3), "assemble": round(t2 - t1, 3)}}
    ncl = [lv["ncells"] for lv in h.levels]
    rt = h.to_layout(b, "column", "tiled")
    zt = torch.empty_like(rt)
    reps = max(5, min(args.steps, 10))
    for form, kw in (("fp64", dict(precision="fp64", krylov="cg")), ("mixed", dict(precision="mixed", krylov="fcg"))):
        kw.update(rtol=1e-8, max_iter=200)
        for _ in range(2):
            _, info = h.solve(b, out=x, **kw)
        total, per = timed_steps(lambda: h.solve(b, out=x, **kw), reps, stream)
        for _ in range(2):
            h.vcycle(rt, precision=form, layout="tiled", out=zt)
        vt, _ = timed_steps(lambda: h.vcycle(rt, precision=form, layout="tiled", out=zt), reps, stream)
        byts = vcycle_bytes(ncl, w["nlayers"], form == "mixed")
        gbs = byts / (vt / reps * 1e-3) / 1e9
        out[form] = {"solves_per_s": round(reps / (total / 1e3), 3), "ms_per_solve": step_stats(per),
                     "iterations": info["iterations"], "true_rel_residual": info["true_rel_residual"],
                     "vcycle": {"ms": round(vt / reps, 4), "model_bytes": int(byts), "GB_s": round(gbs, 1),
                                "frac_of_hbm_peak": round(gbs / hbm, 4)}}
    h.close()
    return out


def run_gpu(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import hmg_inputs as gi
    import paper_1605_00492_gb300 as hmg
    w = gi.WORKLOADS[args.workload]
    r, nz, L = w["refinement"], w["nlayers"], w["nlevels"]
    # ---- setup, timed apart from the solves (the paper's t_setup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = hmg.Hierarchy(r, nz, L)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    h.assemble()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    setup = {"build_hierarchy_s": round(t1 - t0, 4), "assemble_s": round(t2 - t1, 4),
             "what": "host mesh and hierarchy generation with its upload; device assembly of every level "
                     "(first call, FP32 copies included)"}
    n = h.ncells
    stream = torch.cuda.current_stream()
    b = torch.tensor(gi.rhs(n), dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    kw64 = dict(precision="fp64", krylov="cg", rtol=1e-8, max_iter=200)
    kwmx = dict(precision="mixed", krylov="fcg", rtol=1e-8, max_iter=200)

    # warm-up; one traced solve per form gives the per-kernel, per-level breakdown
    for _ in range(args.warmup):
        h.solve(b, out=x, **kw64)
    h.profile_start()
    _, info64 = h.solve(b, out=x, **kw64)
    br64 = h.profile_stop()
    for _ in range(args.warmup):
        h.solve(b, out=x, **kwmx)
    h.profile_start()
    _, infomx = h.solve(b, out=x, **kwmx)
    brmx = h.profile_stop()
    (dom_k, dom_l), _ = max(br64.items(), key=lambda kv: kv[1][1])
    for _ in range(args.warmup):
        h.solve(b, out=x, **kw64)

    # ---- timed region: K FP64 solves, nothing traced (each solve is one
    # device-side CG loop); clocks sampled by nvidia-smi meanwhile
    launches0 = h.launch_count()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        clk.mark(True)
        elapsed_ms, per64 = timed_steps(lambda: h.solve(b, out=x, **kw64), args.steps, stream)
        clk.mark(False)
    barrier(world)
    launches = h.launch_count() - launches0
    _, info = h.solve(b, out=x, **kw64)
    x64 = x.clone()
    elapsed_ms = max_over_ranks(elapsed_ms, world, dev)
    clocks = clk.summary()
    ms64 = elapsed_ms / args.steps
    value = world * args.steps / (elapsed_ms / 1e3)

    # ---- the dominant kernel, traced live over K more solves (after the
    # timed region, so that tracing does not perturb the headline)
    h.profile_start(kernels=[dom_k], levels=[dom_l])
    traced_ms, _ = timed_steps(lambda: h.solve(b, out=x, **kw64), args.steps, stream)
    dom_stats = h.profile_stop()

    # ---- the FP64 pipe's throughput on this device (the roof of the FP64 kernels)
    fp64_probe = h.measure_fp64_rate()

    # ---- mixed form, same protocol (no tracing)
    for _ in range(3):
        h.solve(b, out=x, **kwmx)
    totmx, permx = timed_steps(lambda: h.solve(b, out=x, **kwmx), args.steps, stream)
    msmx = max_over_ranks(totmx, world, dev) / args.steps
    _, infomx = h.solve(b, out=x, **kwmx)
    err_mx = float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))

    # ---- V-cycle alone (tiled layout, no conversions), both forms
    hbm, hbm_src = measured_peaks()
    ncells_levels = [lv["ncells"] for lv in h.levels]
    rt = h.to_layout(b, "column", "tiled")
    zt = torch.empty_like(rt)
    vc = {}
    for form in ("fp64", "mixed"):
        for _ in range(3):
            h.vcycle(rt, precision=form, layout="tiled", out=zt)
        reps = max(10, args.steps)
        vt, _ = timed_steps(lambda: h.vcycle(rt, precision=form, layout="tiled", out=zt), reps, stream)
        ms = vt / reps
        byts = vcycle_bytes(ncells_levels, nz, form == "mixed")
        gbs = byts / (ms * 1e-3) / 1e9
        vc[form] = {"ms": round(ms, 4), "model_bytes": int(byts), "GB_s": round(gbs, 1),
                    "frac_of_hbm_peak": round(gbs / hbm, 4)}

    # ---- velocity-pressure system (Sec. 4.1): GMRES(30) with the Schur-complement
    # preconditioner (Sec. 4.2), to the paper's 1e-5, right-hand side (M2~ R_U, M3 R_P)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    vp = None if args.no_vp else velocity_pressure_section(h, args, world, dev, stream, ev0, ev1)

    # ---- next-to-lowest order (Table "GridSetup": 5,120 columns x 64 layers,
    # 5 levels counting the p-coarsened one), GMRES(30) to the paper's 1e-5
    nlo = nlo_section(args, world, dev, stream, hbm) if not args.no_nlo else None

    # ---- end to end: host buffers through the C ABI (H2D + solve + D2H)
    e2e = None
    if not args.no_e2e:
        bh = b.cpu().pin_memory()
        xh = torch.empty_like(bh).pin_memory()
        for _ in range(2):
            h.solve_host(bh, xh, **kw64)
        tot_e2e, per_e2e = timed_steps(lambda: h.solve_host(bh, xh, **kw64), args.steps, stream)
        ms_e2e = max_over_ranks(tot_e2e, world, dev) / args.steps
        e2e = {"value": round(world / (ms_e2e / 1e3), 3), "unit": UNIT, "h2d_bytes_per_step": int(n * 8),
               "d2h_bytes_per_step": int(n * 8), "ms_per_step": round(ms_e2e, 4),
               "ms_per_step_stats": step_stats(per_e2e)}

    # ---- the horizontal domain decomposition of Sec. 5 emulated on this GPU:
    # K parts with real halo exchanges (pack, segment moves, unpack) before
    # every pass that reads neighbour columns, the coarsest level gathered
    part = None
    if not args.no_extra:
        part = {"what": "FP64 PCG solves of the same problem on K parts of one GPU (hmg_partition); the halo "
                        "exchange's share from one traced solve"}
        for K in (2, 4):
            h.partition(K)
            for _ in range(2):
                _, ik = h.solve(b, out=x, **kw64)
            reps = max(5, min(args.steps, 20))
            totk, perk = timed_steps(lambda: h.solve(b, out=x, **kw64), reps, stream)
            h.profile_start()
            h.solve(b, out=x, **kw64)
            brk = h.profile_stop()
            halo_ms = sum(t for (k, _), (_, t) in brk.items() if k == "halo")
            all_ms = sum(t for _, (_, t) in brk.items())
            part[f"K{K}"] = {"solves_per_s": round(reps / (totk / 1e3), 3), "ms_per_solve": step_stats(perk),
                             "iterations": ik["iterations"], "halo_share_of_traced_time": round(halo_ms / all_ms, 4)}
        h.partition(1)

    # ---- the other workloads: r3x16 latency, r5x64a adjoint, r7x128 both forms
    small = None if args.no_extra else small_config_section(args, dev, stream)
    adjoint = None if args.no_extra else adjoint_section(args, dev, stream)
    large = None if (args.no_extra or args.no_large) else large_config_section(args, dev, stream, hbm)

    # ---- roofline of the dominant kernel
    cnt, tot = dom_stats.get((dom_k, dom_l), (0, 0.0))
    n_l = ncells_levels[dom_l]
    per_cell_b = kernel_bytes_per_cell(dom_k, 8, nz)
    avg_ms = tot / max(cnt, 1)
    gbs = per_cell_b * n_l / (avg_ms * 1e-3) / 1e9
    tflops = KERNEL_FLOPS[dom_k] * n_l / (avg_ms * 1e-3) / 1e12
    t_hbm = per_cell_b * n_l / (hbm * 1e9)
    t_alu = KERNEL_FLOPS[dom_k] * n_l / (FP64_PEAK_TFLOPS * 1e12)
    if t_alu > t_hbm:
        roof = {"bound": "alu", "achieved": round(tflops, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                "peak_source": "derived FP64 FMA rate (152 SM x 4 x 32 lanes / 64 cycles x 2 x 2.07 GHz)",
                "peak_probe_TFLOP_s": round(fp64_probe, 4),
                "frac_of_probe": round(tflops / fp64_probe, 4) if fp64_probe > 0 else None,
                "hbm_achieved_GB_s": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}
    else:
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(gbs / hbm, 4), "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)"}
    roof.update({"kernel": f"{dom_k}@level{dom_l}", "launches": cnt, "avg_us": round(avg_ms * 1e3, 2),
                 "timing": (f"CUDA events around each launch of the kernel inside the captured iteration graphs of "
                            f"{args.steps} FP64 solves traced right after the timed region "
                            f"({round(traced_ms / args.steps, 4)} ms per traced solve)"),
                 "bytes_per_launch": int(per_cell_b * n_l), "flops_per_launch": int(KERNEL_FLOPS[dom_k] * n_l),
                 "traffic": args.traffic if args.traffic is not None else
                 (TRAFFIC_SWEEP_L0_R6X64 if (args.workload == "r6x64" and (dom_k, dom_l) == ("sweep", 0)) else None)})

    def breakdown(br):
        return {f"{k}@{lvl}": {"launches": c, "ms": round(t, 3)} for (k, lvl), (c, t) in sorted(br.items())}

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms64, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args.workload),
        "ms_per_step_stats": step_stats(per64),
        "iterations": info["iterations"], "true_rel_residual": info["true_rel_residual"],
        "setup": setup,
        "mixed": {"solves_per_s": round(world / (msmx / 1e3), 3), "ms_per_solve": round(msmx, 4),
                  "ms_per_solve_stats": step_stats(permx),
                  "iterations": infomx["iterations"], "true_rel_residual": infomx["true_rel_residual"],
                  "rel_l2_vs_fp64_solution": err_mx,
                  "krylov": "flexible CG", "dtype": "f32 cycle / f64 Krylov + coarsest"},
        "partition_emulated": part,
        "r3x16": small,
        "r5x64a_adjoint": adjoint,
        "r7x128": large,
        "vcycle": vc,
        "velocity_pressure": vp,
        "nlo": nlo,
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "breakdown_fp64_one_solve": breakdown(br64),
        "useful_bandwidth_fp64": useful_bandwidth(br64, ncells_levels, nz, hbm),
        "breakdown_mixed_one_solve": breakdown(brmx),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_subprocess(args.workload, args.oracle_iterations)
    if rank == 0:
        print(json.dumps(out), flush=True)
    h.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------- reference arm

def oracle_vcycle_primitives(ops, get_rhs, omega=0.8, nu_pre=2, nu_post=2, n_coarse=2):
    """One oracle V-cycle as a list of its primitive calls.

    Calling the returned callables in order performs, with the oracle's own
    routines (multigrid.smooth / restrict / prolong, the sparse H^ product),
    exactly what multigrid.vcycle(ops, get_rhs()) does, in the same order;
    the result is then in u[0].  Returns (calls, u).
    """
    import numpy as np
    from oracle import multigrid
    L = len(ops)
    u = [None] * L
    rhs = [None] * L

    def zero(l):
        return lambda: u.__setitem__(l, np.zeros_like(rhs[l]))

    def smooth(l):
        return lambda: u.__setitem__(l, multigrid.smooth(ops[l], u[l], rhs[l], omega))

    def restrict(l):
        return lambda: rhs.__setitem__(l + 1, multigrid.restrict(rhs[l] - ops[l].H @ u[l], ops[l + 1].ncols,
                                                                 ops[l].nlayers))

    def prolong(l):
        return lambda: u.__setitem__(l, u[l] + multigrid.prolong(u[l + 1], ops[l + 1].ncols, ops[l].nlayers))

    calls = [lambda: rhs.__setitem__(0, get_rhs())]
    for l in range(L - 1):
        calls.append(zero(l))
        calls += [smooth(l)] * nu_pre
        calls.append(restrict(l))
    calls.append(zero(L - 1))
    calls += [smooth(L - 1)] * n_coarse
    for l in range(L - 2, -1, -1):
        calls.append(prolong(l))
        calls += [smooth(l)] * nu_post
    return calls, u


def oracle_pcg_primitives(ops, b, state=None):
    """The oracle's PCG iterations as an endless stream of primitive calls:
    yields (index within the iteration, calls per iteration, callable).
    `state` (optional dict) receives the iterates x, r, p."""
    import numpy as np
    st = state if state is not None else {}
    st.update({"r": b.copy(), "x": np.zeros_like(b), "p": None, "rz": None})

    def krylov_update(u):
        def f():
            z = u[0]
            rz = float(np.dot(st["r"], z))
            st["p"] = z.copy() if st["p"] is None else z + (rz / st["rz"]) * st["p"]
            st["rz"] = rz
            q = ops[0].H @ st["p"]
            alpha = rz / float(np.dot(st["p"], q))
            st["x"] = st["x"] + alpha * st["p"]
            st["r"] = st["r"] - alpha * q
        return f

    while True:
        calls, u = oracle_vcycle_primitives(ops, lambda: st["r"])
        calls.append(krylov_update(u))
        for i, fn in enumerate(calls):
            yield i, len(calls), fn


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import hmg_inputs as gi
    from oracle import helmholtz, mesh
    w = gi.WORKLOADS[args.workload]
    ms = mesh.hierarchy(w["refinement"], w["nlevels"])
    prm = helmholtz.Params(refinement=w["refinement"], nlayers=w["nlayers"])
    ops = helmholtz.assemble_hierarchy(ms, prm)
    b = gi.rhs(ops[0].ncells)
    stream = oracle_pcg_primitives(ops, b)
    durations = {}

    def run(count):
        for _ in range(count):
            i, P, fn = next(stream)
            t = time.perf_counter()
            fn()
            durations.setdefault(i, []).append(time.perf_counter() - t)
        return P

    # calibrate one iteration, then size each step so that all K + W steps
    # take about REFERENCE_BUDGET_S, covering every primitive at least once.
    t0 = time.perf_counter()
    P = run(1)
    P = run(P - 1)
    t_iter = time.perf_counter() - t0
    per_prim = t_iter / P
    chunk = int(max(-(-P // args.steps), min(P, REFERENCE_BUDGET_S / ((args.steps + args.warmup) * per_prim))))
    chunk = max(chunk, 1)
    for _ in range(args.warmup):
        run(chunk)
    durations.clear()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run(chunk)
    total = time.perf_counter() - t0
    iter_s = sum(statistics.mean(durations[i]) for i in range(P) if i in durations)
    covered = sum(1 for i in range(P) if i in durations)
    value = 1.0 / (iter_s * (ORACLE_ITERATIONS + 1))
    sample = (f"each step: {chunk} of the {P} primitive calls (line relaxation, residual+restriction, "
              f"prolongation, CG update) of one oracle PCG iteration of the {args.workload} FP64 solve; "
              f"iteration time = sum of the mean time of each primitive ({covered}/{P} observed); "
              f"solves/s = 1 / ({ORACLE_ITERATIONS + 1} x iteration time: {ORACLE_ITERATIONS} iterations + the "
              "initial V-cycle); NumPy/SciPy, one thread")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(args.workload),
           "seconds_per_pcg_iteration": round(iter_s, 4),
           "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-nlo", action="store_true", help="skip the next-to-lowest-order section")
    ap.add_argument("--no-vp", action="store_true", help="skip the lowest-order velocity-pressure section")
    ap.add_argument("--no-extra", action="store_true", help="skip the r3x16, r5x64a and r7x128 sections")
    ap.add_argument("--no-large", action="store_true", help="skip the r7x128 section")
    ap.add_argument("--oracle-iterations", type=int, default=8)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.warmup < 3 and args.oracle_sample is None:
        ap.error("--warmup must be >= 3")
    if args.oracle_sample:
        sec, setup = oracle_sample(args.oracle_sample, args.oracle_iterations)
        print(json.dumps({"seconds": sec, "setup_s": setup}))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
