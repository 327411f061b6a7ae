"""Benchmark of the HGKS step on GB300: cell-updates/s on the Taylor-Green
vortex 256^3 in FP64 (Ma 0.1, Re 1600, Pr 0.72, power-law viscosity,
CFL 0.5), synthetic data (the exact-average TGV initial field).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 256]

Prints one JSON line (rank 0).  Besides the FP64 headline (`value`, its
roofline and an end-to-end figure through host buffers) the line carries:
  mixed    - the same workload in mixed precision, with its error against
             the FP64 run and a roofline against the FP32 pipe, and the
             HGKS_MIXED_T64 variant's cost and error (t64_variant);
  batched  - 64 Taylor-Green problems on uneven grids, stepped one by one and
             as one batch (--batch-steps, default 50), FP64 and mixed;
  serve    - the first --serve-requests (default 100) requests of the seeded
             500-request stream through the continuous-batching serve loop;
  cpu_baseline - the CPU oracle on bounded samples (TGV 64^3 and 32^3).
With N > 1 (torchrun, one process per GPU) every rank advances its own
independent replica (the slab decomposition is host logic tested on CPU
ranks; one GPU per run here); value is the total over ranks and the time is
the maximum over ranks.

--histories K runs K steps in FP64 and in mixed precision from the same
field instead and prints the statistics after every step (--case tgv or
channel).

--impl reference times the CPU oracle (test infrastructure, the paper's
method written out plainly in C) on this machine's host cores, on a bounded
sample of the same workload: the same Taylor-Green vortex on a 32^3 grid,
whose per-cell work equals that of the 256^3 grid.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GAMMA = 1.4
MA, RE, PR, OMEGA, CFL = 0.1, 1600.0, 0.72, 0.7, 0.5
METRIC = "cell-updates/s TGV 256^3 FP64 vs mixed at stated error; serve p50/p99 ms"
# DRAM bytes per face of one k_flux launch (dram__bytes_read.sum +
# dram__bytes_write.sum, mean of the 30 k_flux launches of an ncu capture of
# `bench.py --n 128 --steps 1 --warmup 3` on the current build: 3219 MB read +
# 244 MB written for 2,113,536 faces), scaled by the faces of a launch.  The
# 128^3 input of the pass (1.9 GB of first-tangential records) is 15x the L2,
# so the per-face figure carries over to 256^3 (at 64^3, where the input is
# only twice the L2, a launch moved 1.02 instead of 1.73 kB per face).
K_FLUX_DRAM_BYTES_PER_FACE = (3219.49e6 + 243.97e6) / 2113536
K_FLUX_TRAFFIC_CURRENT = True
# the same for k_flux_mx (2010 MB read + 170 MB written per 128^3 launch,
# mean of 24 launches of the current build)
K_FLUX_MX_DRAM_BYTES_PER_FACE = (2009.60e6 + 170.24e6) / 2113536
K_FLUX_MX_TRAFFIC_CURRENT = True
# executed FP64 flops per k_flux face (2 DFMA + DMUL + DADD thread
# instructions from sass__thread_inst_executed_true_per_opcode, ncu capture of
# `bench.py --n 48` on the current build), for the roofline's note
K_FLUX_EXECUTED_FP64_FLOPS_PER_FACE = 14345
# GB300 FP32 (non-tensor) peak: 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Table 3 of the paper: 256^3 TGV, FP64, Tesla V100, 11.697 h for 20 t_c at dt = 8.925e-4
PAPER_V100_CUPS = 256 ** 3 * (20.0 / 8.925e-4) / (11.697 * 3600.0)


def tgv_kwargs():
    p0 = 1.0 / (GAMMA * MA * MA)
    return dict(visc=(1, 1.0 / RE, p0, OMEGA), Pr=PR, gamma=GAMMA)


def workload_config(n):
    import paper_2207_01173_gb300 as hg
    fp = hg.footprint_bytes((n, n, n))
    return {"workload": "Taylor-Green vortex %d^3 FP64, Ma %.1f, Re %d, Pr %.2f, power-law viscosity "
                        "(omega %.1f), CFL %.1f" % (n, MA, RE, PR, OMEGA, CFL),
            "grid": [n, n, n], "precision": "fp64",
            "l2": "no flush: inputs larger than L2 (each state buffer %.0f MB, %.1f GB of device buffers per "
                  "step against a 129 MB L2)" % (5 * (n + 6) ** 3 * 8 / 1e6, fp / 1e9),
            "data": "synthetic exact-average TGV initial field"}


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline / reference arm)
# --------------------------------------------------------------------------
def oracle_rate(steps, n=32):
    """cell-updates/s of the CPU oracle on the n^3 TGV (same per-cell work as
    256^3), `steps` full steps after one untimed step."""
    from oracle import ref
    s = ref.RefSolver((n, n, n), **{k: v for k, v in tgv_kwargs().items()})
    s.init_tgv(MA, 1.0, 1.0)
    s.step(1, CFL)
    t0 = time.perf_counter()
    s.step(steps, CFL)
    el = time.perf_counter() - t0
    s.close()
    return n ** 3 * steps / el, el


def oracle_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else os.cpu_count()


def host_cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline line."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    rate, el = oracle_rate(args.warmup, args.ref_n)  # warm-up steps (timed region below)
    rate, el = oracle_rate(args.steps, args.ref_n)
    cores = oracle_threads()
    sample = "TGV %d^3 (same Ma, Re, Pr, viscosity law and CFL; per-cell work equals the %d^3 grid's): " \
             "%d warm-up steps on a first solver, then 1 untimed and %d timed steps on a second" \
             % (args.ref_n, args.n, args.warmup, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.n),
            "cpu_baseline": {"value": rate, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                             "cpu_model": host_cpu_model(), "sample": sample},
            "e2e": {"value": rate, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# the GPU path
# --------------------------------------------------------------------------
def batched_leg(hg, args, stream):
    """Many small problems: 64 Taylor-Green vortices on uneven grids advanced
    together (one persistent kernel per pass over all of them, one CUDA graph
    per step), against the same problems stepped one after another through
    hgks_step.  Both arms start from the same initial fields and take the
    same steps, so their final states must agree bit for bit."""
    import torch
    from paper_2207_01173_gb300 import workloads

    probs = workloads.batch_tgv_problems()
    cells = sum(int(np.prod(n)) for n, _, _ in probs)
    out = {"workload": "64 Taylor-Green vortices, each grid dimension drawn from {24,32,48,64,96}, Ma U[0.1,0.5], "
                       "Re log-U[400,3200], seed 64, CFL %.1f" % CFL,
           "problems": len(probs), "cells": cells}
    for prec, name, steps in ((hg.FP64, "fp64", args.batch_steps), (hg.MIXED, "mixed", args.batch_steps)):
        solvers = [hg.Solver(n, precision=prec, **workloads.tgv_solver_kwargs(Ma, Re)) for n, Ma, Re in probs]

        def init():
            for sv, (n, Ma, Re) in zip(solvers, probs):
                sv.init_tgv(Ma, 1.0, 1.0)

        # one problem after another through hgks_step
        init()
        for sv in solvers:
            sv.step(1, CFL)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for sv in solvers:
            sv.step(steps, CFL)
        ev1.record(stream)
        torch.cuda.synchronize()
        seq_ms = ev0.elapsed_time(ev1)
        seq_states = [sv.get_state() for sv in solvers]

        # the same, batched
        init()
        b = hg.Batch(solvers)
        tune_ms = b.tune(CFL)
        b.step(1, CFL)
        with ClockSampler(torch.cuda.current_device()) as clk:
            b.step(steps, CFL)
        info = b.info()
        b.close()
        bat_ms = info["last_ms"]
        same = all(np.array_equal(sv.get_state(), q) for sv, q in zip(solvers, seq_states))
        del seq_states
        for sv in solvers:
            sv.close()
        out[name] = {"value": cells * steps / (bat_ms * 1e-3), "unit": "cell-updates/s", "steps": steps,
                     "warmup": 1, "ms_per_step": bat_ms / steps,
                     "sequential_value": cells * steps / (seq_ms * 1e-3),
                     "speedup_vs_sequential": seq_ms / bat_ms,
                     "bitwise_equal_to_sequential": bool(same),
                     "tiles_chosen": {k: info[k] for k in ("tile_cells", "tile_normal", "tile_tan1", "tile_sweep",
                                                           "tile_normal_mx")},
                     "tuned_passes_ms": tune_ms, "launches_per_step": info["launches_per_step"],
                     "gpu_launches": info["launches_per_step"] * steps, "tiles": info["tiles"],
                     "clocks": clk.summary()}
    return out


def serve_leg(hg, args, capacity):
    """The serving workload: a seeded Poisson stream of Taylor-Green and
    channel solves in mixed precision, served by the continuous-batching loop
    with admission by device footprint.  The arrival rate is 0.8 of the
    measured capacity (cell-updates/s of the batched mixed path) divided by
    the mean work per request of the whole 500-request stream; the first
    --serve-requests requests of that stream are served."""
    import torch
    from paper_2207_01173_gb300 import workloads
    from paper_2207_01173_gb300.serve import CudaEngine, Server

    stream = workloads.serve_requests()
    mean_work = float(np.mean([workloads.request_work(r) for r in stream]))
    rate = 0.8 * capacity / mean_work
    reqs = [dict(r, t=r["arrival"] / rate) for r in stream[:args.serve_requests]]
    free, _ = torch.cuda.mem_get_info()
    budget = int(min(0.8 * free, args.serve_budget_gb * 2 ** 30))
    eng = CudaEngine(precision=hg.MIXED, cfl=CFL)
    srv = Server(eng, budget, max_chunk=args.serve_chunk, policy=args.serve_policy, age_s=args.serve_age)
    with ClockSampler(torch.cuda.current_device()) as clk:
        res, summ = srv.run(reqs)
    eng.close()
    summ.update(workload="Poisson stream (seed 500) of Taylor-Green (60%%, N in {32..192}) and channel (40%%, "
                         "N in {64,96,128}) solves of 20-200 steps, mixed precision; first %d of 500 requests"
                % len(reqs),
                arrival_rate_per_s=rate, capacity_cell_updates_per_s=capacity, mean_work_cell_updates=mean_work,
                max_chunk=args.serve_chunk, policy=args.serve_policy, age_s=args.serve_age,
                batch_rebuilds=eng.rebuilds,
                batch_rebuild_create_s=eng.rebuild_create_s,
                batch_rebuild_capture_s=eng.rebuild_capture_s,
                clocks=clk.summary(),
                latency_percentiles="numpy linear interpolation over completed requests")
    return summ


def run_histories(args):
    """Statistics after every step of a run in FP64 and in mixed precision
    from the same initial field: the statistical error of the mixed path over
    a longer run.  --case tgv: the Taylor-Green vortex (E_k, enstrophy,
    dissipation); --case channel: the channel (E_k, mean wall shear).  Prints
    one JSON line."""
    import torch
    import paper_2207_01173_gb300 as hg
    from paper_2207_01173_gb300 import workloads
    n, K = args.n, args.histories
    keys = ("Ek", "enstrophy", "eps_com") if args.case == "tgv" else ("Ek", "wall_shear", "mass")
    hist = {}
    for name, prec in (("fp64", hg.FP64), ("mixed", hg.MIXED)):
        if args.case == "tgv":
            sv = hg.Solver((n, n, n), precision=prec, **tgv_kwargs())
            sv.init_tgv(MA, 1.0, 1.0)
        else:
            sv = hg.Solver((n, n, n), precision=prec, **workloads.channel_solver_kwargs())
            sv.init_channel(0.5, 0.1, 2800)
        rows = []
        prof, nprof = None, 0
        t0 = time.perf_counter()
        for i in range(K):
            sv.step(1, CFL)
            st = sv.stats()
            rows.append([st["t"]] + [st[k] for k in keys])
            if args.case == "channel" and i >= K - K // 4:
                # mean streamwise velocity profile <rho u> / <rho> over x and z,
                # averaged over the last quarter of the run (a host diagnostic)
                q = sv.get_state()
                u = q[1].mean(axis=(0, 2)) / q[0].mean(axis=(0, 2))
                prof = u if prof is None else prof + u
                nprof += 1
        torch.cuda.synchronize()
        hist[name] = (np.array(rows), time.perf_counter() - t0, None if prof is None else prof / nprof)
        sv.close()
    a, b = hist["fp64"][0], hist["mixed"][0]
    rel = np.abs(b[:, 1:] - a[:, 1:]) / np.abs(a[:, 1:])
    every = max(1, K // 20)
    workload = (workload_config(n)["workload"] if args.case == "tgv" else
                "channel %d^3, Ma_b 0.5, Re_b 2800, 2pi x 2 x pi, tanh-stretched y (b 2), isothermal walls, body "
                "force (180/2800)^2, 10%% seeded velocity noise, CFL %.1f" % (n, CFL))
    line = {"mode": "histories", "case": args.case, "workload": workload, "steps": K,
            "max_rel_diff": {k: float(rel[:, i].max()) for i, k in enumerate(keys)},
            "t_end": {"fp64": float(a[-1, 0]), "mixed": float(b[-1, 0])},
            "wall_s": {"fp64": hist["fp64"][1], "mixed": hist["mixed"][1]},
            "history": [dict({"step": i + 1, "t": float(a[i, 0])},
                             **{k: float(a[i, j + 1]) for j, k in enumerate(keys)},
                             **{k + "_rel": float(rel[i, j]) for j, k in enumerate(keys)})
                        for i in range(every - 1, K, every)]}
    if args.case == "channel":
        pa, pb = hist["fp64"][2], hist["mixed"][2]
        line["mean_u_profile"] = {
            "averaged_over_steps": K // 4,
            "max_rel_diff": float(np.abs(pb - pa).max() / np.abs(pa).max()),
            "y_index_every_8": {"fp64": [float(v) for v in pa[::8]], "mixed": [float(v) for v in pb[::8]]}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    # CPU baseline first (no GPU context yet), rank 0 only, N = 1 only
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # two samples: 32^3 (its 2.2 MB state buffers sit in the host caches)
        # and 64^3 (14 MB state buffers, 0.5 GB of face records per sweep,
        # beyond the caches, like 256^3); the 64^3 rate is the reported value
        rate32, el32 = oracle_rate(args.cpu_steps, args.ref_n)
        rate64, el64 = oracle_rate(1, 64)
        cpu_baseline = {"value": rate64, "unit": "cell-updates/s", "cores": oracle_threads(), "kind": "oracle",
                        "cpu_model": host_cpu_model(),
                        "sample": "TGV 64^3, 1 step after 1 untimed (%.1f s; per-cell work equals the %d^3 "
                                  "grid's, working set beyond the host caches); beside it TGV %d^3, %d steps "
                                  "after 1 untimed (%.1f s)" % (el64, args.n, args.ref_n, args.cpu_steps, el32),
                        "value_32": rate32, "ratio_64_over_32": rate64 / rate32}

    torch.cuda.set_device(local_rank)
    import paper_2207_01173_gb300 as hg
    from paper_2207_01173_gb300.decomp import max_over_ranks

    n = args.n
    cells = n ** 3
    solver = hg.Solver((n, n, n), **tgv_kwargs())
    solver.init_tgv(MA, 1.0, 1.0)
    # the end-to-end leg's pinned host buffers, allocated once up front as an
    # application would: allocated after the other legs' large host arrays
    # came and went, the same buffers copied 10-20x slower
    q_host = torch.empty((5, n, n, n), dtype=torch.float64).pin_memory()
    out_host = torch.empty_like(q_host).pin_memory()
    stream = torch.cuda.current_stream()
    model = hg.flop_model((n, n, n))
    fp64_peak = hg.fp64_probe() if rank == 0 else None

    def timed_run(sv):
        for _ in range(args.warmup):
            sv.step_timed(CFL)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        with ClockSampler(local_rank) as clk:
            ev0.record(stream)
            for _ in range(args.steps):
                times.append(sv.step_timed(CFL))
            ev1.record(stream)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
        ms = max_over_ranks(ev0.elapsed_time(ev1), device="cuda")
        return ms, times, clk.summary()

    ms, times, clocks = timed_run(solver)
    ms_per_step = ms / args.steps
    value = world * cells * args.steps / (ms * 1e-3)
    q64 = solver.get_state()
    s64 = solver.stats()

    # the mixed-precision path on the same workload, same number of steps from
    # the same initial field: throughput and its error against the FP64 run
    mixed = None
    if not args.no_mixed:
        mx = hg.Solver((n, n, n), precision=hg.MIXED, **tgv_kwargs())
        mx.init_tgv(MA, 1.0, 1.0)
        ms_mx, times_mx, clocks_mx = timed_run(mx)
        qmx = mx.get_state()
        smx = mx.stats()
        mx.close()
        scale = np.abs(q64).reshape(5, -1).max(axis=1)
        scale[1:4] = scale[1:4].max()
        inst = float((np.abs(qmx - q64).reshape(5, -1).max(axis=1) / scale).max())
        del qmx
        mixed = {"value": world * cells * args.steps / (ms_mx * 1e-3), "unit": "cell-updates/s",
                 "ms_per_step": ms_mx / args.steps,
                 "speedup_vs_fp64": ms / ms_mx,
                 "kernel_ms_per_step": {k: sum(t[k] for t in times_mx) / args.steps
                                        for k in ("ghost_ms", "dt_ms", "normal_ms", "tan1_ms", "flux_ms",
                                                  "update_ms", "other_ms")},
                 "error_vs_fp64": {"steps": args.warmup + args.steps,
                                   "instantaneous_rel_linf": inst,
                                   "Ek_rel": abs(smx["Ek"] - s64["Ek"]) / abs(s64["Ek"]),
                                   "enstrophy_rel": abs(smx["enstrophy"] - s64["enstrophy"]) / abs(s64["enstrophy"])},
                 "clocks": clocks_mx,
                 "gpu_launches": sum(t["launches"] for t in times_mx)}
        # the flux pass against the FP32 pipe: the method's algorithmic flops
        # per face (the same formulas the FP64 count covers; the mixed path
        # carries some values as float-float pairs on top) over the measured
        # k_flux_mx launch time
        fl_ms = sum(t["flux_ms"] for t in times_mx) / sum(t["flux_launches"] for t in times_mx)
        fl_flops = model["flux_per_face"] * (n + 1) * n * n
        ach = fl_flops / (fl_ms * 1e-3) / 1e12
        mixed["roofline"] = {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": ach / FP32_PEAK_TFLOPS, "traffic": K_FLUX_MX_DRAM_BYTES_PER_FACE * (n + 1) * n * n if K_FLUX_MX_TRAFFIC_CURRENT else None,
                             "traffic_note": "ncu DRAM bytes per k_flux_mx launch on TGV 128^3 scaled by faces",
                             "kernel": "k_flux_mx",
                             "peak_note": "FP32 FMA peak from unit counts and clock: 152 SMs x 128 lanes x 2 "
                                          "flops x 2.07 GHz",
                             "algorithmic_flops_per_launch": fl_flops, "avg_launch_ms": fl_ms}
        # the same with the Maxwellian temperature, collision time and time
        # coefficients of every Gauss point in FP64 (HGKS_MIXED_T64): its cost
        # and its error beside the FP32 split's
        if not args.no_t64:
            m64 = hg.Solver((n, n, n), precision=hg.MIXED_T64, **tgv_kwargs())
            m64.init_tgv(MA, 1.0, 1.0)
            ms_t, times_t, clocks_t = timed_run(m64)
            qt = m64.get_state()
            st_t = m64.stats()
            m64.close()
            inst_t = float((np.abs(qt - q64).reshape(5, -1).max(axis=1) / scale).max())
            del qt
            mixed["t64_variant"] = {
                "value": world * cells * args.steps / (ms_t * 1e-3), "unit": "cell-updates/s",
                "ms_per_step": ms_t / args.steps, "cost_vs_mixed": ms_t / ms_mx,
                "flux_ms_per_step": sum(t["flux_ms"] for t in times_t) / args.steps,
                "error_vs_fp64": {"steps": args.warmup + args.steps, "instantaneous_rel_linf": inst_t,
                                  "Ek_rel": abs(st_t["Ek"] - s64["Ek"]) / abs(s64["Ek"]),
                                  "enstrophy_rel": abs(st_t["enstrophy"] - s64["enstrophy"]) / abs(s64["enstrophy"])},
                "clocks": clocks_t}
    del q64

    # end to end through the public API with host buffers: pinned H2D of the
    # state, one step, D2H of the resulting state, every step
    solver.get_state(q_host)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    phase = {"h2d_ms": 0.0, "step_ms": 0.0, "d2h_ms": 0.0}
    with ClockSampler(local_rank) as clk_e2e:
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ta = time.perf_counter()
            solver.set_state(q_host)
            tb = time.perf_counter()
            solver.step(1, CFL)
            tc = time.perf_counter()
            solver.get_state(out_host)
            td = time.perf_counter()
            phase["h2d_ms"] += (tb - ta) * 1e3 / e2e_steps
            phase["step_ms"] += (tc - tb) * 1e3 / e2e_steps
            phase["d2h_ms"] += (td - tc) * 1e3 / e2e_steps
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, device="cuda")
    e2e_value = world * cells * e2e_steps / e2e_s
    stats = solver.stats()

    solver.close()
    batched = None if args.no_batched else batched_leg(hg, args, stream)
    serve = None
    if rank == 0 and args.serve_requests > 0:
        cap = args.serve_capacity or (batched["mixed"]["value"] if batched else (mixed["value"] if mixed else value))
        serve = serve_leg(hg, args, cap)

    if rank != 0:
        return 0
    # dominant kernel: the flux pass (six launches per step)
    flux_ms = sum(t["flux_ms"] for t in times)
    flux_launches = sum(t["flux_launches"] for t in times)
    launches = sum(t["launches"] for t in times)
    kernel_ms = {k: sum(t[k] for t in times) / args.steps
                 for k in ("ghost_ms", "dt_ms", "normal_ms", "tan1_ms", "flux_ms", "update_ms", "other_ms")}
    faces_per_launch = (n + 1) * n * n
    flops_per_launch = model["flux_per_face"] * faces_per_launch
    achieved = flops_per_launch / (flux_ms / flux_launches * 1e-3) / 1e12
    peak = 1.25  # nominal dense FP64, TFLOP/s
    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_V100_CUPS, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(n), parallelism=("replicas%d" % world) if world > 1 else "single-gpu"),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": K_FLUX_DRAM_BYTES_PER_FACE * faces_per_launch if K_FLUX_TRAFFIC_CURRENT else None,
                     "traffic_note": "ncu DRAM bytes per k_flux launch on TGV 128^3 (mean of 30 launches, current "
                                     "build) scaled by faces to one 256^3 launch", "kernel": "k_flux",
                     "peak_note": "nominal GB300 dense FP64 (1.25 TFLOP/s); measured FP64 FMA probe %.3f TFLOP/s"
                                  % fp64_peak,
                     "algorithmic_flops_per_launch": flops_per_launch,
                     "flops_per_face": model["flux_per_face"], "faces_per_launch": faces_per_launch,
                     "avg_launch_ms": flux_ms / flux_launches,
                     "executed_frac": K_FLUX_EXECUTED_FP64_FLOPS_PER_FACE * faces_per_launch
                                      / (flux_ms / flux_launches * 1e-3) / 1e12 / peak,
                     "flops_note": "hgks_flop_model counts the written arithmetic of the current flux; "
                                   "divisions and special functions count 1 each, so ncu's executed FP64 "
                                   "flops per face (%d at 48^3) are above the count and frac sits below "
                                   "the FP64 pipe's 87 %% utilisation" % K_FLUX_EXECUTED_FP64_FLOPS_PER_FACE},
        "step_flops": model["per_step"],
        "step_tflops": model["per_step"] / (ms_per_step * 1e-3) / 1e12,
        "kernel_ms_per_step": kernel_ms,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": 5 * cells * 8,
                "d2h_bytes_per_step": 5 * cells * 8, "steps": e2e_steps,
                "phase_ms_per_step": phase, "clocks": clk_e2e.summary()},
        "cpu_baseline": cpu_baseline,
        "mixed": mixed,
        "batched": batched,
        "serve": serve,
        "final_stats": {"t": stats["t"], "step": stats["step"], "Ek": stats["Ek"], "enstrophy": stats["enstrophy"]},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--ref-n", type=int, default=32)
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-t64", action="store_true", help="skip the HGKS_MIXED_T64 variant of the mixed leg")
    ap.add_argument("--batch-steps", type=int, default=50)
    ap.add_argument("--serve-requests", type=int, default=100)
    ap.add_argument("--serve-budget-gb", type=float, default=96.0)
    ap.add_argument("--serve-chunk", type=int, default=8)
    ap.add_argument("--histories", type=int, default=0,
                    help="instead of the benchmark: K steps in FP64 and mixed, statistics after each")
    ap.add_argument("--case", choices=["tgv", "channel"], default="tgv", help="problem of --histories")
    ap.add_argument("--serve-policy", choices=["fair", "srpt"], default="srpt")
    ap.add_argument("--serve-age", type=float, default=10.0,
                    help="srpt aging: remaining work is divided by 1 + wait / this many seconds")
    ap.add_argument("--serve-capacity", type=float, default=0.0,
                    help="cell-updates/s that sets the arrival rate (default: the measured batched mixed rate)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        world = max(world, 1)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.histories > 0:
        return run_histories(args)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
