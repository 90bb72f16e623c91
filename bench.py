"""Benchmark of the GB300 JFNK hot path.

Headline: the batched workload, the largest that runs on one GPU.  A step is one complete
Newton-Krylov solve (residual, Jv, FP32 multigrid V-cycle, loose GMRES(30) with an FP32 basis
and FP64 Arnoldi arithmetic, Newton with line search) of 512 independent 3-D linear-elastic
boxes (7.63 M cells in total, cell counts log-uniform in 1k-64k, 4:1:1 shape, +-15 % node
perturbation, random E, nu and end traction) held in one index space, each problem from u = 0
to its own |R| <= 1e-8 |R(0)|.  The metric is Jv cell-updates per second of whole-solve time:
sum over problems of cells x Jacobian-vector products, over the solve time.

The same line carries sub-records of the other workloads (`workloads`): the 80,000-cell
cantilever (200x20x20) and the 262,144-cell neo-Hookean beam (256x32x32, 10 load steps),
with the same metric, and the served request stream (Poisson arrivals, 2k-1M cells, 70 %
Hooke / 30 % neo-Hookean) with solves/s and p50/p99 latency per arrival rate, against the
same requests solved one after another, in FP64 and in mixed precision, and served in FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c4|c2|c3|c6] [--serve] [--no-sub]

N > 1 (torchrun, one rank per GPU): independent replicas of the same solve per rank (the
method is not sharded; no collective on the data path); value = all ranks' cell-updates /
the slowest rank's time.  `--impl reference` times the FP64 CPU oracle (the baseline of this
project) on all host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Jv cell-updates/s"
UNIT = "cell-updates/s"
HBM_PEAK_FALLBACK = 6800.0
# FP64 ALU roof: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": HBM_PEAK_FALLBACK}, "fallback"


def workload_case(name="c2"):
    from paper_2502_17217_gb300 import inputs as I
    if name == "c3":
        return I.case_nh_beam()
    if name == "c4":
        return [I.case_batch_member(*x, index=k) for k, x in enumerate(I.batch_sizes())]
    if name == "c6":
        return I.case_dynamic_beam(24, 240, 24)[0]
    return I.case_cantilever(200, 20, 20, (1.0, 0.1, 0.1), perturb=0.15, seed=2)


DRAM_BYTES_PER_LAUNCH = {"c2": {"update": 16.04e6, "mdot": 16.57e6, "flux": 30.90e6}}
# the batched workload: DRAM bytes per evaluated cell (read + write, one ncu capture on its first
# 96 problems, 1.31 M cells, every row evaluated), scaled by the cells a launch evaluates; the
# cell-sum pass has changed since that capture (one thread per cell for all three components),
# so it has no figure
DRAM_BYTES_PER_CELL = {"c4": {"pc_mg": 615.0, "flux": 506.8, "grad": 243.8}}
# FP64 thread instructions (DFMA + DADD + DMUL) per launch, from ncu's per-cycle instruction
# rates x elapsed cycles of the same capture (k_flux: 47 per internal face, 231,600 of them)
FP64_INSTR_PER_LAUNCH = {"c2": {"flux": 10.90e6}}
# the same count per internal Hooke face (10.90 M / 231,600), for the all-Hooke batch, whose
# face pass is counted as internal faces x this (its displacement faces, under 3 %, left out)
FP64_INSTR_PER_HOOKE_FACE = 10.90e6 / 231600
FP64_ISSUE_PEAK_GINSTR = 152 * 2 * 2.07  # thread instructions per ns: 152 SM x 2 per clock x 2.07 GHz
KRYLOV = ("loose GMRES(30) keeping 2 corrections across restarts (Sec. 4.2), right-preconditioned, "
          "FP32 basis, FP64 Arnoldi arithmetic")
WORKLOADS = {
    "c2": {"workload": "cantilever_200x20x20_perturbed15", "cells": 80000, "dofs": 240000,
           "law": "linear elastic (E=200 GPa, nu=0.3)", "pc": "multigrid V-cycle (FP32)",
           "krylov": KRYLOV, "tolerance": "|R|/|R0| < 1e-8",
           "eta": 1e-3, "jv_eps": "1e-7 (1+|u|)/|v|", "load_steps": 1},
    "c3": {"workload": "neo_hookean_beam_256x32x32", "cells": 262144, "dofs": 786432,
           "law": "neo-Hookean total Lagrangian (mu=0.38 MPa, kappa=8.3 MPa)", "pc": "multigrid V-cycle (FP32)",
           "krylov": KRYLOV, "tolerance": "|R|/|R0| < 1e-8 per load step",
           "eta": 1e-3, "jv_eps": "1e-7 (1+|u|)/|v|", "load_steps": 10},
    "c6": {"workload": "dynamic_column_24x240x24_case6", "cells": 138240, "dofs": 414720,
           "law": "neo-Hookean (E=15.293 MPa, nu=0.3), rho=1000 kg/m^3, sudden traction (50,50,0) kPa on the upper face",
           "pc": "multigrid V-cycle (FP32)", "krylov": KRYLOV,
           "tolerance": "|R|/|R0| < 1e-8 per time step", "eta": 1e-3, "jv_eps": "1e-7 (1+|u|)/|v|", "load_steps": 1,
           "time_steps_per_bench_step": 10, "dt_s": 1e-3, "integrator": "BDF2 with the Taylor predictor (Sec. 2.3, 3.2)"},
    "c4": {"workload": "batch_512_boxes_logU_1k_64k", "cells": None, "dofs": None,
           "law": "linear elastic, E~U(1,300) GPa, nu~U(0.2,0.45)", "pc": "multigrid V-cycle (FP32)",
           "krylov": KRYLOV + ", per problem", "tolerance": "|R|/|R0| < 1e-8 per problem",
           "eta": 1e-3, "jv_eps": "1e-7 (1+|u_p|)/|v_p| per problem", "load_steps": 1},
}
WORKLOAD = WORKLOADS["c4"]


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join(tempfile.gettempdir(), f"jfnk_bench_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        self.f = None
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if self.f:
                self.f.close()
                try:
                    os.remove(self.path)
                except OSError:
                    pass
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            lines = fh.readlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else 0.0,
                             parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r[2] > 200.0] or rows
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in load:
            for nm, val in zip(names, r[3:]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(load),
                "power_w_max": max(r[2] for r in rows)}


# flops (FMA = 2) and algorithmic bytes per launch of the residual passes, from the mesh
def kernel_costs(case):
    m = case.mesh
    nc, ni = m.n_cells, m.n_internal
    nd = sum(p.size for p in m.patches if p.bc == 0)
    slots = 2 * ni  # internal face sides
    flux_flops = ni * 77 + nd * 53
    grad_flops = slots * 21
    # algorithmic bytes: each input read once, each output written once
    n_tensors = 1 if case.material.law == 0 else 2  # the gradient, and the traction operator for TL laws
    flux_bytes = (ni + nd) * (11 * 8 + 4) + ni * 4 + n_tensors * 9 * 8 * nc + 2 * 3 * 8 * nc + (ni + nd) * 3 * 8
    grad_bytes = slots * (4 + 3 * 8) + nc * 3 * 8 + nc * 9 * 8
    finish_bytes = (ni + nd) * 3 * 8 + ni * 4 + nc * (3 * 8 + 3 * 8 + 3 * 8 + 4 * 4)
    finish_flops = (2 * ni + nd) * 3 + nc * 9
    return {"flux": (flux_flops, flux_bytes), "grad": (grad_flops, grad_bytes), "finish": (finish_flops, finish_bytes)}


def vcycle_bytes(levels, sweeps, s=4, tv=4):
    """Algorithmic bytes of one V-cycle over the hierarchy `levels` (rows, operator and
    prolongation entries per level), each input of each kernel read once and each output
    written once, three right-hand sides, values of s bytes, int32 indices:
      * per level above the coarsest, 2 x sweeps + 1 operator passes (the smoothing sweeps
        down and up and the residual): x, b, D^-1, the off-diagonal entries with their column
        indices, the row pointers, and the written vector;
      * restriction: r, the entries of P^T with indices, row pointers, the coarse b;
      * prolongation: the coarse x, the entries of P with indices, row pointers, x read and
        written;
      * the coarsest level: its dense inverse, b and x;
      * the finest level's input (the FP32 Krylov vector, tv bytes) and output (z, FP64)."""
    if not levels:
        return 0.0
    n0 = levels[0]["rows"]
    tot = 3.0 * tv * n0 + 24.0 * n0
    for l in range(len(levels) - 1):
        L = levels[l]
        n, nnz, npz, nco = L["rows"], L["nnz_a"], L["nnz_p"], levels[l + 1]["rows"]
        op = 3 * s * n + 3 * s * n + s * n + (nnz - n) * (s + 4) + 4 * n + 3 * s * n
        tot += (2 * sweeps + 1) * op
        tot += 3 * s * n + npz * (s + 4) + 4 * nco + 3 * s * nco
        tot += 3 * s * nco + npz * (s + 4) + 4 * n + 6 * s * n
    c = levels[-1]["rows"]
    tot += float(c) * c * s + 6 * s * c
    return tot


def aggregate_ranks(t_ms, units, device):
    """Replicas: the job's time is the slowest rank's, its work the sum over ranks (every rank
    gets both).  Works with any torch.distributed backend (gloo tensors on the CPU)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def make_solver(workload, dev, members=0, **extra):
    """The solver (or batch) of a workload with the benchmark's options; returns (s, case).
    members > 0 keeps the first `members` problems of the batched workload (profiling runs)."""
    from paper_2502_17217_gb300 import jfnk
    case = workload_case(workload)
    if workload == "c4" and members > 0:
        case = case[:members]
    opts = dict(device=dev.index, pc=jfnk.PC_MG, precision=jfnk.PREC_MIXED, newton_rtol=1e-8, gmres_restart=30,
                gmres_eta=1e-3, **extra)
    if workload == "c4":
        return jfnk.Batch(case, **opts), case[0], opts
    if workload == "c6":
        return jfnk.Solver.from_case(case, density=1000.0, dt=1e-3, **opts), case, opts
    return jfnk.Solver.from_case(case, **opts), case, opts


def run_ours(workload, steps, warmup, rank=0, world=1, shapes="", profile=True, e2e_steps=None, segregated=False):
    """Times `steps` solves of `workload` after `warmup` untimed ones (CUDA events on the
    launching stream, L2 flushed before each); with `profile`, per-kernel event times from
    extra solves; then the end-to-end figure through the C ABI with host buffers."""
    import torch
    import __graft_entry__ as g
    g.build()
    dev = torch.device("cuda", rank % max(1, torch.cuda.device_count()))
    torch.cuda.set_device(dev)
    s, case, opts = make_solver(workload, dev)
    nc = s.nc
    load_steps = WORKLOADS[workload]["load_steps"]
    s.setup()
    if shapes:
        s.set_tuning(*[int(v) for v in shapes.split(",")])
    # the library launches on the caller's stream: a dedicated stream, current for every call,
    # so the CUDA events below sit on the launching stream
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    u0 = torch.zeros((nc, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step():
        if workload == "c6":  # ten time steps, continuing the motion
            u, st, rc, _ = s.solve_dynamic(WORKLOADS["c6"]["time_steps_per_bench_step"])
        else:
            u, st, rc = s.solve(u0, load_steps=load_steps)
        if rc != 0:
            raise RuntimeError(f"solve failed: status {rc}, rel res {st.final_rel_res:.3e}")
        return st

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = s.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    jv_total = 0
    stats = []
    with ClockSampler(dev.index) as clk:
        for k in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            ev[k][0].record(stream)
            st = step()
            ev[k][1].record(stream)
            torch.cuda.synchronize()
            jv_total += jv_cell_updates(s, st, workload) / nc
            stats.append(st)
    launches = s.launch_count() - launches0
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        t_ms, jv_total = aggregate_ranks(t_ms, jv_total, dev)
    value = nc * jv_total / (t_ms / 1e3)
    kt = {}
    prof_work = {"arnoldi_cols": 0.0, "reorth_cols": 0.0, "its": 0.0, "reorth_its": 0.0, "res_cells": 0.0, "vc_cells": 0.0}
    if profile:
        # per-kernel times: the same solve with CUDA events on the launch stream around every
        # kernel (events cannot sit inside the captured iteration graph, so these steps launch
        # the kernels directly)
        s.profile(True)
        s.profile_reset()
        for _ in range(max(1, min(steps, 2))):
            flush.zero_()
            torch.cuda.synchronize()
            pst = step()
            for key, val in arnoldi_work(s, pst, workload).items():
                prof_work[key] += val
        torch.cuda.synchronize()
        s.profile(False)
        for name in ("grad", "flux", "finish", "mdot", "update", "pc_mg"):
            ms, n = s.profile_get(name)
            kt[name] = {"ms": ms, "launches": n}
        # the steps inside the V-cycle from one more solve with their own events (which would
        # inflate the whole-V-cycle time above)
        s.profile(True, detail=True)
        s.profile_reset()
        flush.zero_()
        torch.cuda.synchronize()
        step()
        torch.cuda.synchronize()
        s.profile(False)
        for name in ("mg_smooth", "mg_resid", "mg_restrict", "mg_prolong", "mg_coarse"):
            ms, n = s.profile_get(name)
            kt[name] = {"ms": ms, "launches": n, "detail_solve": True}
    # end to end through the C ABI with host buffers (copies inside the timed region)
    n_e2e = steps if e2e_steps is None else max(1, min(steps, e2e_steps))
    u_host = np.zeros((nc, 3))
    if workload != "c6":
        s.solve(u_host, load_steps=load_steps)
    t0 = time.perf_counter()
    jv_e2e = 0
    for _ in range(n_e2e):
        if workload == "c6":  # the call returns the displacement to host memory
            u, st, rc, _ = s.solve_dynamic(WORKLOADS["c6"]["time_steps_per_bench_step"])
        else:
            u, st, rc = s.solve(u_host, load_steps=load_steps)
        jv_e2e += jv_cell_updates(s, st, workload) / nc
    e2e_s = time.perf_counter() - t0
    e2e_value = nc * jv_e2e / e2e_s * world
    seg = None
    if segregated and workload == "c2":
        seg = segregated_comparison(case, opts, stream)
    elif segregated and workload == "c6":
        seg = segregated_comparison_dynamic(case, dict(opts, density=1000.0, dt=1e-3), stream)
    levels = s.mg_hierarchy()
    torch.cuda.set_stream(torch.cuda.default_stream(dev))
    return {"value": value, "t_ms": t_ms, "stats": stats, "kernels": kt, "launches": launches, "clocks": clk.summary(),
            "e2e": e2e_value, "e2e_steps": n_e2e, "case": case, "solver": s, "nc": nc, "prof_work": prof_work,
            "tuning": s.tuning(), "segregated": seg, "levels": levels, "sweeps": s.options.mg_smooth_sweeps}


def segregated_comparison_dynamic(case, opts, stream, n_steps=5):
    """Case 6 comparison: the first n_steps time steps from rest, each solved by the
    Newton-Krylov method and by the segregated method (same residual, J~, multigrid)."""
    import torch
    from paper_2502_17217_gb300 import jfnk
    out = {"time_steps": n_steps, "rtol": opts.get("newton_rtol")}
    for name, seg in (("jfnk", False), ("segregated", True)):
        s = jfnk.Solver.from_case(case, **opts)
        s.setup()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        u, st, rc, _ = s.solve_dynamic(n_steps, raise_on_fail=False, segregated=seg)
        b.record(stream)
        torch.cuda.synchronize()
        out[name] = {"solve_time_s": a.elapsed_time(b) / 1e3, "status": rc, "outer_its": st.newton_its,
                     "krylov_or_cg_its": st.gmres_its, "steps_done": st.load_steps_done}
        s.close()
    out["jfnk_speedup"] = out["segregated"]["solve_time_s"] / out["jfnk"]["solve_time_s"]
    return out


def segregated_comparison(case, opts, stream, rtol=1e-6, max_outer=60000):
    """The paper's comparison (Sec. 4): the same problem solved by the Newton-Krylov path and
    by the segregated quasi-Newton method of Sec. 3.1 (same residual, J~ and multigrid), both
    to the paper's |R|/|R0| < 1e-6, timed with CUDA events on the launch stream."""
    import torch
    from paper_2502_17217_gb300 import jfnk
    o = dict(opts, newton_rtol=rtol, seg_max_outer=max_outer)
    s = jfnk.Solver.from_case(case, **o)
    s.setup()
    out = {"rtol": rtol}
    s.solve(raise_on_fail=False)  # warm-up of the Newton-Krylov path (graph capture)
    for name, fn in (("jfnk", s.solve), ("segregated", s.solve_segregated)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        u, st, rc = fn(raise_on_fail=False)
        b.record(stream)
        torch.cuda.synchronize()
        out[name] = {"solve_time_s": a.elapsed_time(b) / 1e3, "status": rc, "outer_its": st.newton_its,
                     "krylov_or_cg_its": st.gmres_its, "final_rel_res": st.final_rel_res}
    out["jfnk_speedup"] = out["segregated"]["solve_time_s"] / out["jfnk"]["solve_time_s"]
    s.close()
    return out


def jv_cell_updates(s, st, workload):
    """Cells x Jacobian-vector products of one solve (a batch: each problem's cells x its own
    products)."""
    if workload == "c4":
        return sum(ps.jv_products * n for ps, n in zip(s.problem_stats(), s.sizes))
    return st.jv_products * s.nc


def arnoldi_work(s, st, workload):
    """Element-weighted Gram-Schmidt work of one solve: sum over iterations of 3 n_p (j + 1),
    the same over the repeated projections, 3 n_p per iteration and per repeated projection."""
    if workload == "c4":
        per = list(zip(s.problem_stats(), s.sizes))
    else:
        per = [(st, s.nc)]
    return {"arnoldi_cols": sum(3 * n * p.arnoldi_cols for p, n in per),
            "reorth_cols": sum(3 * n * p.reorth_cols for p, n in per),
            "its": sum(3 * n * p.gmres_its for p, n in per),
            "reorth_its": sum(3 * n * p.reorth_its for p, n in per),
            # cells x residual evaluations (Jv, Newton and line-search residuals) and cells x
            # V-cycles (one per Jacobian product of the right-preconditioned Arnoldi process)
            # of the problems that took part in them
            "res_cells": sum(n * p.residual_evals for p, n in per),
            "vc_cells": sum(n * p.jv_products for p, n in per)}


MG_ORACLE = dict(theta=0.4, coarse_max=1000, smoothed=True, sweeps=2)  # the solver's default hierarchy options


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _oracle_case(workload, index):
    from paper_2502_17217_gb300 import inputs as I
    if workload == "c4":
        return I.case_batch_member(*I.batch_sizes()[index], index=index)
    return workload_case(workload)


def oracle_job(job):
    """One oracle worker: loose GMRES(30, 2) cycles with the oracle's FP64 V-cycle (the
    solver's hierarchy options) on the first Newton step of one problem of the workload, for
    about `seconds`.  Returns (cell-updates, iterations, seconds, cells)."""
    import oracle as O
    workload, index, seconds = job
    case = _oracle_case(workload, index)
    o = O.Oracle.from_case(case)
    steps = WORKLOADS[workload]["load_steps"]
    if steps > 1:
        o.set_load_factor(1.0 / steps)
    o.mg_setup(**MG_ORACLE)
    nc = case.mesh.n_cells
    u = np.zeros((nc, 3))
    R = o.residual(u)
    its_total, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        _, _, its, _ = o.lgmres(u, -R, m=30, aug=2, eta=1e-3, max_restarts=1, pc=O.PC_MG, R_u=R)
        its_total += max(1, its)
    dt = time.perf_counter() - t0
    return nc * its_total, its_total, dt, nc


def oracle_pool():
    """Worker processes for the oracle on every host core, started with spawn (no CUDA state
    is inherited)."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(processes=os.cpu_count() or 1)


def _members_sample(workload, n, step=0):
    """Seeded sample of n problems of the workload (for the batch: member indices)."""
    if workload != "c4":
        return [0] * n
    from paper_2502_17217_gb300 import inputs as I
    r = I.splitmix64_uniform(97 + step, n, key=5)
    return [int(x * 512) for x in r]


def cpu_baselines(workload, pool, seconds_1=12.0, seconds_all=10.0):
    """The oracle on one core (one worker busy) and on all cores (one worker per core, each on
    its own problem of the workload), as cell-updates/s."""
    ncores = os.cpu_count() or 1
    mean_member = None
    if workload == "c4":
        from paper_2502_17217_gb300 import inputs as I
        sizes = [nx * ny * nz for nx, ny, nz, *_ in I.batch_sizes()]
        mean_member = int(np.argmin(np.abs(np.array(sizes) - np.mean(sizes))))
    cu, its, dt, nc = pool.apply(oracle_job, ((workload, mean_member or 0, seconds_1),))
    one = {"value": cu / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{its} oracle loose-GMRES(30, 2) iterations (Jv + FP64 V-cycle + Gram-Schmidt) of the first "
                     f"Newton step of one {nc}-cell problem, {dt:.1f} s",
           "cpu_model": cpu_model()}
    jobs = [(workload, k, seconds_all) for k in _members_sample(workload, ncores)]
    res = pool.map(oracle_job, jobs)
    tot = sum(x[0] for x in res)
    wall = max(x[2] for x in res)
    allc = {"value": tot / wall, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": f"{ncores} processes, one per core, each {seconds_all:.0f} s of oracle loose-GMRES(30, 2) "
                      f"iterations on its own problem of the workload ({sum(x[1] for x in res)} iterations, "
                      f"{sum(x[3] for x in res)} cells in all)",
            "cpu_model": one["cpu_model"]}
    return {"cpu_baseline": allc, "cpu_baseline_1core": one}


def reference_line(args):
    """The reference arm: the oracle as it stands, on all host cores, on the workload's
    problems; each step a bounded sample (one worker per core, a few seconds each)."""
    pool = oracle_pool()
    ncores = os.cpu_count() or 1
    try:
        for w in range(args.warmup):
            pool.map(oracle_job, [(args.workload, k, 1.0) for k in _members_sample(args.workload, ncores, 1000 + w)])
        vals, t_steps, its = [], [], 0
        for k in range(args.steps):
            res = pool.map(oracle_job, [(args.workload, m, 3.0) for m in _members_sample(args.workload, ncores, k)])
            wall = max(x[2] for x in res)
            vals.append(sum(x[0] for x in res) / wall)
            t_steps.append(wall)
            its += sum(x[1] for x in res)
    finally:
        pool.close()
        pool.join()
    value = float(np.mean(vals))
    sample = (f"per step {ncores} processes (one per core), each ~3 s of oracle loose-GMRES(30, 2) iterations with the "
              f"FP64 V-cycle on the first Newton step of its own problem of the workload; {its} iterations in all")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(t_steps)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOADS[args.workload], sample=sample),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_for_ncu(args):
    """Untimed solves of the workload, for an ncu capture of the same kernels."""
    import torch
    import __graft_entry__ as g
    g.build()
    dev = torch.device("cuda", 0)
    extra = dict(autotune=0) if args.shapes else {}
    s, case, _ = make_solver(args.workload, dev, members=args.members, **extra)
    if args.shapes:  # with --shapes the autotuner is off, so a capture's launch count starts at the solve
        s.set_tuning(*[int(v) for v in args.shapes.split(",")])
    for _ in range(args.warmup + args.steps):
        u, st, rc = s.solve(load_steps=WORKLOADS[args.workload]["load_steps"])
        if rc != 0:
            raise SystemExit(f"solve failed: {rc}")
    torch.cuda.synchronize()
    print(json.dumps({"ncu_driver": True, "gmres_its": st.gmres_its, "newton_its": st.newton_its}))


def fp64_issue(workload, kernel, launch_s, fp64_measured_tflops, evaluated=1.0):
    """The dominant kernel against the FP64 issue rate rather than the flop rate: a DADD or
    DMUL takes an issue slot for one flop, so a kernel whose mix has them cannot reach the flop
    roof even with the pipe always busy.  None where no instruction count was captured.
    `evaluated`: the mean fraction of the batch's union a launch evaluates (problems out of
    the Arnoldi iteration sit its passes out)."""
    n = FP64_INSTR_PER_LAUNCH.get(workload, {}).get(kernel)
    source = "ncu sm__sass_thread_inst_executed_op_{dfma,dadd,dmul} rates x cycles, one capture"
    if n is None and workload == "c4" and kernel == "flux":
        n = FP64_INSTR_PER_HOOKE_FACE * sum(c.mesh.n_internal for c in workload_case("c4")) * evaluated
        source = ("47.06 FP64 instructions per internal Hooke face (ncu, 80k-cell cantilever) x the internal "
                  f"faces a launch evaluates (mean {evaluated:.3f} of the union)")
    if n is None:
        return None
    ach = n / launch_s / 1e9
    measured = fp64_measured_tflops * 1e3 / 2  # the measuring kernel issues FMAs only
    return {"instr_per_launch": n, "achieved_ginstr_s": ach, "peak_ginstr_s": FP64_ISSUE_PEAK_GINSTR,
            "frac": ach / FP64_ISSUE_PEAK_GINSTR, "frac_of_measured": ach / measured, "source": source}


def serving_record(args):
    """Config 5: Poisson arrivals of solve requests (cells log-uniform 2k-1M, 70% Hooke / 30%
    neo-Hookean with 2 load steps).  Served with continuous admission in mixed precision at each
    arrival rate, and in FP64 at the highest rate; against the same requests solved one after
    another in FP64 and in mixed precision (set-up included, as for a served request), so that
    the gain splits into precision (sequential FP64 -> sequential mixed) and concurrency
    (sequential mixed -> served mixed)."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2502_17217_gb300 import inputs as I, jfnk, serving
    torch.cuda.set_device(0)
    reqs_def = I.serving_requests(args.requests, seed=5)
    cases = [c for c, _ in reqs_def]
    steps = [st for _, st in reqs_def]
    mixed = dict(pc=jfnk.PC_MG, precision=jfnk.PREC_MIXED, newton_rtol=1e-8)
    fp64 = dict(pc=jfnk.PC_MG, precision=jfnk.PREC_FP64, newton_rtol=1e-8)

    def sequential(opts):
        t0 = time.perf_counter()
        us, lat = [], []
        for c, st in reqs_def:
            t1 = time.perf_counter()
            s = jfnk.Solver.from_case(c, **opts)
            u, stt, rc = s.solve(load_steps=st, raise_on_fail=False)
            us.append(u)
            s.close()
            lat.append(time.perf_counter() - t1)
        return us, time.perf_counter() - t0, lat

    plain_u, t_seq, lat_seq = sequential(fp64)
    _, t_seq_mixed, _ = sequential(mixed)

    def served(rate, opts, mode="contexts", setup_ahead=0):
        reqs, wall, srv = serving.serve_stream(cases, rate_per_s=rate, seed=int(rate), load_steps=steps, max_slots=args.slots,
                                               mode=mode, setup_ahead=setup_ahead, **opts)
        summ = serving.summarize(reqs, wall)
        err = max(float(np.linalg.norm(r.u - up) / max(np.linalg.norm(up), 1e-300)) if r.u is not None else float("inf")
                  for r, up in zip(reqs, plain_u))
        summ.update(max_concurrent=srv.max_concurrent, max_solving=srv.max_solving, max_rel_diff_vs_sequential_fp64=err,
                    setup_s_total=float(sum(getattr(r, "t_setup", 0.0) for r in reqs)),
                    wait_s_total=float(sum(getattr(r, "t_wait", 0.0) for r in reqs)),
                    solve_s_total=float(sum(getattr(r, "t_solve", 0.0) for r in reqs)))
        return summ

    rates = {}
    rate_list = [float(x) for x in args.rates.split(",")]
    for rate in rate_list:
        rates[str(int(rate))] = served(rate, mixed)
    lockstep = {str(int(rate)): served(rate, mixed, mode="lockstep") for rate in rate_list}
    served_fp64 = served(max(rate_list), fp64)
    best = max(v["solves_per_s"] for v in rates.values())
    seq = len(reqs_def) / t_seq
    seq_mixed = len(reqs_def) / t_seq_mixed
    return {"metric": "served solves/s", "value": best, "unit": "solves/s", "higher_is_better": True,
            "config": {"workload": "serving_poisson_logU_2k_1M_70lin_30nh", "requests": args.requests,
                       "cells_total": int(sum(c.mesh.n_cells for c in cases)),
                       "served": f"continuous admission by HBM footprint, {args.slots} slots, one context and stream per request, "
                                 "MG FP32 + FP32 basis (mixed)",
                       "baseline": "the same requests solved one after another (set-up included)"},
            "rates": rates, "lockstep_rates": lockstep, "served_fp64_at_max_rate": served_fp64,
            "modes": {"rates": f"contexts: one context and stream per request, up to {args.slots} at once",
                      "lockstep_rates": "lockstep: queued requests with the same load steps concatenated into one "
                                        f"batch (one index space and iteration graph), up to {args.slots} batches at once"},
            "sequential_fp64_solves_per_s": seq, "sequential_fp64_p50_latency_s": float(np.percentile(lat_seq, 50)),
            "sequential_mixed_solves_per_s": seq_mixed,
            "speedup_vs_sequential_fp64": best / seq,
            "speedup_split": {"precision (sequential mixed / sequential FP64)": seq_mixed / seq,
                              "concurrency (served mixed / sequential mixed)": best / seq_mixed,
                              "concurrency in FP64 (served FP64 / sequential FP64)": served_fp64["solves_per_s"] / seq}}


def serving_line(args):
    rec = serving_record(args)
    rec.update(n_gpus=1, steps=len(rec["rates"]), warmup=0, scaling="weak", vs_baseline=None, dtype="f64",
               data="synthetic")
    return rec


def kernel_totals(r, workload):
    """Algorithmic (flops, bytes) of every profiled kernel over the profiled solves."""
    case = r["case"]
    costs = kernel_costs(case) if workload != "c4" else None
    if costs is None:  # batch: costs of the whole union mesh
        costs = {k: (0, 0) for k in ("grad", "flux", "finish")}
        for cs in workload_case("c4"):
            for k, (f_, b_) in kernel_costs(cs).items():
                costs[k] = (costs[k][0] + f_, costs[k][1] + b_)
    # residual passes per launch x launches; Gram-Schmidt from the counted work (FMA = 2
    # flops; FP32 basis reads, FP64 w read and written); the V-cycle's bytes from its
    # hierarchy (FP32 arithmetic: no FP64 flops)
    w = r["prof_work"]
    kt = r["kernels"]
    nc = r["nc"]
    if workload == "c4":
        # a batch's problems outside the Arnoldi iteration skip its passes: the work is the
        # union's cost per cell x the cells of the evaluations each problem took part in
        units = {k: w["res_cells"] / nc for k in ("grad", "flux", "finish")}
        vc_units = w["vc_cells"] / nc
    else:
        units = {k: kt[k]["launches"] for k in ("grad", "flux", "finish")}
        vc_units = kt["pc_mg"]["launches"]
    tot = {k: (costs[k][0] * units[k], costs[k][1] * units[k]) for k in ("grad", "flux", "finish")}
    tot["mdot"] = (2 * (w["arnoldi_cols"] + w["its"]), 4 * w["arnoldi_cols"] + 8 * w["its"])
    tot["update"] = (2 * (w["arnoldi_cols"] + 2 * w["reorth_cols"]),
                     4 * (w["arnoldi_cols"] + w["reorth_cols"]) + 16 * (w["its"] + w["reorth_its"]))
    tot["pc_mg"] = (0.0, vcycle_bytes(r["levels"], r["sweeps"]) * vc_units)
    return tot


WORK_UNITS = ("algorithmic flops / bytes over the kernel's CUDA-event time in the profiled solves: residual passes "
              "per cell-evaluation x (problem cells x residual evaluations it took part in), V-cycles per fine cell x "
              "(problem cells x Jacobian products), Gram-Schmidt per basis element projected; per-launch figures are "
              "those totals over the launches")


def build_roofline(r, workload):
    """The dominant kernel (largest measured time) against its binding roof: FP64 issue for
    the residual and Gram-Schmidt kernels, HBM for the FP32 V-cycle; the others alongside."""
    from paper_2502_17217_gb300 import jfnk as _j
    peaks, src = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", HBM_PEAK_FALLBACK)
    kt = r["kernels"]
    tot = kernel_totals(r, workload)
    top = max(tot, key=lambda k: kt[k]["ms"])
    t_s = kt[top]["ms"] / 1e3
    launches = max(1, kt[top]["launches"])
    flops, nbytes = tot[top]
    fp64_measured = _j.measure_fp64_rate(0)
    traffic = DRAM_BYTES_PER_LAUNCH.get(workload, {}).get(top)
    per_cell = DRAM_BYTES_PER_CELL.get(workload, {}).get(top)
    if per_cell is not None:
        cells = r["prof_work"]["vc_cells"] if top == "pc_mg" else r["prof_work"]["res_cells"]
        traffic = per_cell * cells / launches
    profiled = sum(kt[q]["ms"] for q in ("grad", "flux", "finish", "mdot", "update", "pc_mg"))
    others = {k: {"tflops": tot[k][0] / (kt[k]["ms"] / 1e3) / 1e12, "gbs": tot[k][1] / (kt[k]["ms"] / 1e3) / 1e9,
                  "hbm_frac": tot[k][1] / (kt[k]["ms"] / 1e3) / 1e9 / hbm_peak,
                  "fp64_frac": tot[k][0] / (kt[k]["ms"] / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                  "share_of_profiled": kt[k]["ms"] / profiled, "launches": kt[k]["launches"]}
              for k in tot if kt[k]["ms"] > 0}
    if top == "pc_mg":
        achieved = nbytes / t_s / 1e9
        return {"kernel": "pc_mg (one V-cycle)", "bound": "hbm", "work_units": WORK_UNITS, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": src, "traffic": traffic,
                "algorithmic_bytes_per_launch": nbytes / launches, "avg_launch_us": t_s / launches * 1e6,
                "fp64_measured_tflops": fp64_measured, "others": others}
    achieved = flops / t_s / 1e12
    return {"kernel": top, "bound": "alu", "work_units": WORK_UNITS, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "fp64_measured_tflops": fp64_measured,
            "frac_of_measured_fp64": achieved / fp64_measured, "traffic": traffic,
            "algorithmic_bytes_per_launch": nbytes / launches,
            "peak_source": "FP64 ALU: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz (recipe nominal 1.25 TFLOP/s)",
            "hbm_achieved_gbs": nbytes / t_s / 1e9, "hbm_peak_gbs": hbm_peak, "hbm_frac": nbytes / t_s / 1e9 / hbm_peak,
            "hbm_peak_source": src, "avg_launch_us": t_s / launches * 1e6,
            "fp64_issue": fp64_issue(workload, top, t_s / launches, fp64_measured,
                                     evaluated=(r["prof_work"]["res_cells"] / r["nc"] / launches) if workload == "c4" else 1.0),
            "others": others}


def sub_record(workload, steps, warmup, segregated=False):
    """A compact record of another workload with the same metric (no per-kernel profile)."""
    r = run_ours(workload, steps, warmup, profile=False, e2e_steps=1, segregated=segregated)
    st = r["stats"]
    rec = {"metric": METRIC, "value": r["value"], "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": r["t_ms"] / steps,
           "config": dict(WORKLOADS[workload], cells=r["nc"], dofs=3 * r["nc"],
                          l2="flushed (256 MB write) before every step"),
           "newton_its": st[-1].newton_its, "gmres_its": st[-1].gmres_its, "jv_products": st[-1].jv_products,
           "final_rel_res": st[-1].final_rel_res, "gpu_launches": r["launches"], "clocks": r["clocks"],
           "e2e": {"value": r["e2e"], "unit": UNIT, "steps": r["e2e_steps"],
                   "h2d_bytes_per_step": 0 if workload == "c6" else 24 * r["nc"], "d2h_bytes_per_step": 24 * r["nc"]}}
    if r["segregated"]:
        rec["vs_segregated"] = r["segregated"]
    r["solver"].close()
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="headline only: no sub-records of the other workloads")
    ap.add_argument("--no-segregated", action="store_true", help="skip the segregated-solver comparison (C2)")
    ap.add_argument("--ncu", action="store_true", help="untimed solves only, for an ncu capture of the same kernels")
    ap.add_argument("--workload", default="c4", choices=["c2", "c3", "c4", "c6"])
    ap.add_argument("--serve", action="store_true", help="config 5 alone: Poisson request stream, served solves/s and p50/p99")
    ap.add_argument("--rates", default="10,30,100,300,1000")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--slots", type=int, default=8, help="serving: requests (or lockstep batches) on the device at once")
    ap.add_argument("--members", type=int, default=0, help="with --ncu and the batched workload: its first N "
                    "problems only (a smaller case for counter captures)")
    ap.add_argument("--e2e-steps", type=int, default=5, help="solves in the end-to-end figure (at most --steps)")
    ap.add_argument("--shapes", default="", help="launch shapes instead of the autotuner's: grad_bs,flux_bs,"
                    "flux_stage,finish_bs,mg_bs (jfnk_set_tuning)")
    args = ap.parse_args()
    if args.serve:
        print(json.dumps(serving_line(args)))
        return
    if args.ncu:
        return run_for_ncu(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_line(args)))
        return
    pool = None
    if rank == 0 and not args.no_cpu_baseline:
        pool = oracle_pool()  # spawn-started worker processes, before the first GPU call
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_ours(args.workload, args.steps, args.warmup, rank, world, shapes=args.shapes, e2e_steps=args.e2e_steps,
                 segregated=(args.workload in ("c2", "c6") and not args.no_segregated))
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    nc = r["nc"]
    st = r["stats"]
    cfg = dict(WORKLOADS[args.workload], cells=nc, dofs=3 * nc, parallelism=f"replicas{world}",
               l2="flushed (256 MB write) before every step", launch_shapes=r["tuning"],
               mg_levels=[lv["rows"] for lv in r["levels"]])
    if args.workload == "c4":
        cfg["problems"] = len(r["solver"].sizes)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["t_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "solve_time_s": r["t_ms"] / args.steps / 1e3,
            "newton_its": st[-1].newton_its, "gmres_its": st[-1].gmres_its, "jv_products": st[-1].jv_products,
            "final_rel_res": st[-1].final_rel_res, "reorth_its": st[-1].reorth_its,
            "roofline": build_roofline(r, args.workload),
            "kernels": r["kernels"],
            "gpu_launches": r["launches"],
            "clocks": r["clocks"],
            "e2e": {"value": r["e2e"], "unit": UNIT, "steps": r["e2e_steps"],
                    "h2d_bytes_per_step": 0 if args.workload == "c6" else 24 * nc, "d2h_bytes_per_step": 24 * nc}}
    if r["segregated"]:
        line["vs_segregated"] = r["segregated"]
    case_for_cpu = r["case"]
    r["solver"].close()
    if pool is not None:
        line.update(cpu_baselines(args.workload, pool))
        pool.close()
        pool.join()
    if not args.no_sub and world == 1:
        subs = {}
        for wl, k_, w_ in (("c2", 5, 3), ("c3", 2, 1)):
            if wl != args.workload:
                subs[wl] = sub_record(wl, k_, w_, segregated=(wl == "c2" and not args.no_segregated))
        subs["c5"] = serving_record(args)
        line["workloads"] = subs
    print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
