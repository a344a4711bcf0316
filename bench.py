#!/usr/bin/env python3
"""Benchmark of the GB300 BP RI-OEDG solver: P2 Euler DG cell-stage updates/s.

Workload (default): the 60-degree double Mach reflection on [0,4]x[0,1], a
1440 x 360 jittered grid split into 1,036,800 triangles, P2, RIOE + BP on,
SSP-RK3 at the optimal-decomposition BP CFL.  One "step" is one SSP-RK3 time
step (3 stages; each stage runs the whole hot path: volume quadrature, edge
LF fluxes, OE statistics, RIOE damping, BP limiter, wave-speed reduction).
value = cells * 3 * steps / time, with the state resident in HBM (the working
set is about 1.7 GB, far above the 129 MB L2, so no L2 flush is needed).

One JSON line is printed by rank 0.  Under torchrun (N > 1) every rank runs
its own replica of the workload on its GPU (independent problems, no
collective on the data path: weak scaling); time is the max over ranks.

--impl reference times the CPU oracle (the repository's plain FP64 C
restatement of the paper) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
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

METRIC = "P2 Euler DG cell-stage updates/s (FP64 vs FP32), HBM GB/s; p50/p99 solve latency"
UNIT = "cell-stage updates/s"

# Algorithmic FP64 work per cell-stage of each kernel kind (P2 interior cell,
# RIOE, limiter on, cell not limited), counted from the kernel source: add /
# sub / mul / division / square root / exponential = 1 flop, fma = 2; a
# compile-time coefficient of 0 costs nothing and one of +-1 a single add; the
# first term into a zero accumulator is one multiply.  k_rk: volume evaluation
# 208, volume fluxes 186, volume accumulation 368, edge terms 529, mass
# inverse and RK combination 106 (mean of the three stages; the first has no
# u_n term), vertex records 269, Hessians 73, block sums 6.  k_stats:
# deviations at the volume points 231, edge OE records 187 per edge x 1.5.
# k_oe_bp: sigma 87, damping 38, limiter at the 11 points 497, traces and
# wave speeds 313 (the nine reciprocal densities from one division and 24
# multiplies); a cell that the bound over the whole cell settles skips the
# 11 points (about 30 flops instead of 497).
ALGO_FLOPS_P2 = {"rk": 1745.0, "stats": 512.0, "oe_bp": 935.0}
# FP64 flops per cell-stage the hardware executed for the same kernels
# (2 DFMA + DMUL + DADD from ncu captures / cells; k_rk: mean of its three
# stages 1896 / 1968 / 1968); division, square root and exp expand into
# DFMA sequences.  None = not re-measured since the kernel last changed.
EXECUTED_FLOPS_P2 = {"rk": 1944.0, "stats": 744.0, "oe_bp": 967.0}
# DRAM bytes (read + write) per launch from the same captures (k_rk: mean of
# its stages 1.599 / 1.808 / 1.808 GB).
TRAFFIC_PER_LAUNCH = {"rk": 1.738e9, "stats": 0.948e9, "oe_bp": 1.301e9}
# Mixed form (P2, FP32 modes 1-5 and FP64 averages: S = 4 x 8 + 4 x 5 x 4 =
# 112 B of state per cell).  Algorithmic HBM bytes per cell-stage of the
# method's three passes, each array element moved once and neighbour data
# taken from L2: the flux pass reads u_n and v and writes u_h (the first
# stage has v = u_n, read once: 2S; the others 3S) plus the geometry it needs
# (FP32 inverse Jacobian 16, normals 24, lengths 12; FP64 |K| and 1/|K| 16;
# neighbour indices 12: G1 = 80 B); the statistics pass reads u_h (S); the
# OE + limiter pass reads u_h and writes u_sigma (2S) plus its geometry
# (normals 24, OE lengths h and 1/h 24, limiter nodes 16, indices 12,
# inverse Jacobian 16: G3 = 92 B).  A launch of the flux kernel
# averages the three stages: (2 + 3 + 3) / 3 S + G1.
S_MIXED_P2 = 112.0
ALGO_BYTES_MIXED_P2 = {"rk": (8.0 / 3.0) * S_MIXED_P2 + 80.0, "stats": S_MIXED_P2,
                       "oe_bp": 2.0 * S_MIXED_P2 + 92.0}
# DRAM bytes per launch of the mixed-form kernels from one ncu capture (k_rk:
# mean of its stages 272 / 394 / 394 B per cell)
TRAFFIC_MIXED_PER_LAUNCH = {"rk": 0.366e9, "stats": 0.120e9, "oe_bp": 0.304e9}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 peak of GB300: 152 SMs x 2 DFMA/clk/SM x 2 flops x 2.07 GHz (the
# recipe's nominal 1.25 TFLOP/s; a DFMA throughput probe measured 1.20 at 2.0 GHz)
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"dg_clocks_rank{index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        loaded = [r for r in rows if r[2] > 300.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def make_workload(name, nx, ny):
    from paper_2409_09620_gb300 import workloads as W
    if name == "dmr":
        return W.dmr_workload(nx=nx, ny=ny, k=2)
    if name == "sedov":
        return W.sedov_workload(n=nx, k=2)
    if name == "vortex":
        return W.vortex_workload(n=nx, k=1)
    raise ValueError(name)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("DG_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def dist_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_rate(wl, steps, max_seconds=30.0):
    """CPU oracle (plain FP64 C, OpenMP over cells) on the host cores."""
    from oracle import oracle as O
    om = O.OracleMesh.from_mesh(wl.mesh)
    u = O.project_workload(om, wl)
    cf = O.config_for(wl)
    t, done, t0 = 0.0, 0, time.perf_counter()
    while done < steps:
        u, t, dt, cnt, rc = om.step(cf, u, t, 1e9)
        done += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    el = time.perf_counter() - t0
    return wl.mesh.nt * 3 * done / el, done, el, O.num_threads()


def cpu_baseline(wl, steps=10, max_seconds=25.0, single_core_seconds=8.0):
    """The oracle timed on every host core (the reported baseline) and on one
    core, on a bounded sample of the workload's steps."""
    from oracle import oracle as O
    rate, done, el, threads = oracle_rate(wl, steps=steps, max_seconds=max_seconds)
    out = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{done} oracle SSP-RK3 step(s) of the full {wl.mesh.nt}-cell workload ({el:.1f} s)"}
    O.set_num_threads(1)
    try:
        r1, d1, e1, _ = oracle_rate(wl, steps=1, max_seconds=single_core_seconds)
    finally:
        O.set_num_threads(threads)
    out["single_core"] = {"value": r1, "unit": UNIT, "cores": 1,
                          "sample": f"{d1} oracle SSP-RK3 step(s) of the same workload ({e1:.1f} s)"}
    return out


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle, each step one SSP-RK3 step of the DMR
    problem on a coarser grid of the same generator, sized so that the run
    stays within a few minutes."""
    if rank != 0:
        return
    from oracle import build as ob
    ob.build()
    total = args.steps + args.warmup
    # about 0.6e6 cell-stage/s per 8 host threads: aim at ~120 s for the whole run
    from oracle import oracle as O
    threads = O.num_threads()
    rate_guess = 0.7e6 * threads / 8.0
    cells_budget = rate_guess * 120.0 / (3.0 * max(total, 1))
    s = max(1, int(math.ceil(math.sqrt(args.nx * args.ny * 2 / max(cells_budget, 2000.0)))))
    nx, ny = max(8, args.nx // s), max(4, args.ny // s)
    wl = make_workload(args.workload, nx, ny)
    om = O.OracleMesh.from_mesh(wl.mesh)
    u = O.project_workload(om, wl)
    cf = O.config_for(wl)
    t = 0.0
    for _ in range(args.warmup):
        u, t, dt, cnt, rc = om.step(cf, u, t, 1e9)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u, t, dt, cnt, rc = om.step(cf, u, t, 1e9)
    el = time.perf_counter() - t0
    value = wl.mesh.nt * 3 * args.steps / el
    sample = (f"{args.steps} oracle SSP-RK3 steps of the same problem on a {nx}x{ny} grid "
              f"({wl.mesh.nt} cells, 1/{s} of the resolution per direction)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded jittered grid, analytic initial state)",
            "config": {"workload": f"dmr{args.nx}x{args.ny}_P2", "cells": args.nx * args.ny * 2, "k": 2,
                       "sample_cells": wl.mesh.nt, "precision": "fp64", "oe": "RI", "bp": "optimal-points"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="dmr", choices=["dmr", "sedov", "vortex"])
    ap.add_argument("--nx", type=int, default=1440)
    ap.add_argument("--ny", type=int, default=360)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=10)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="precision of the primary timed run")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-cfl-gain", action="store_true")
    ap.add_argument("--no-paper-meshes", action="store_true",
                    help="skip the forward-facing-step and wedge meshes")
    ap.add_argument("--no-scalar", action="store_true", help="skip the scalar conservation laws")
    ap.add_argument("--to-t-end", type=float, default=0.2,
                    help="run the DMR to this end time (0 = skip): both forms on a 480 x 120 grid, the mixed "
                         "form on the main grid")
    ap.add_argument("--to-t-end-grid", default="480x120",
                    help="grid of the FP64 / mixed pair run to the end time")
    ap.add_argument("--to-t-end-transmissive", action="store_true",
                    help="also run the main grid with a transmissive right side (the cell-average exterior) "
                         "to the end time in the mixed form")
    ap.add_argument("--to-t-end-full-fp64", action="store_true",
                    help="also run FP64 on the main grid to the end time (about 16 minutes at 1440 x 360)")
    ap.add_argument("--sedov-t-end", type=float, default=0.0,
                    help="run the Sedov blast (256 x 256, P2, FP64) to this end time (0 = skip)")
    ap.add_argument("--serve-requests", type=int, default=16,
                    help="requests per serving run (the serving configuration's size and end-time ranges)")
    ap.add_argument("--serve-rates", default="1,4,16",
                    help="Poisson arrival rates (requests/s) swept in the mixed form")
    ap.add_argument("--serve-steps-per-tick", type=int, default=16)
    ap.add_argument("--serve-fp64-requests", type=int, default=6,
                    help="requests of the FP64 serving run at the highest rate (0 = skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        barrier(world)
        return

    import torch
    torch.cuda.set_device(local)
    from paper_2409_09620_gb300 import build as pbuild
    pbuild.build()
    from paper_2409_09620_gb300 import native as N

    wl = make_workload(args.workload, args.nx, args.ny)
    nt = wl.mesh.nt
    mesh = N.Mesh.from_mesh(wl.mesh)
    u0 = N.initial_state(mesh, wl)
    peaks, peak_src = load_peaks()

    def timed(precision):
        solver = N.Solver(mesh, N.config_for(wl, precision=precision), u0)
        stream = torch.cuda.ExternalStream(solver.stream)
        solver.advance_async(args.warmup)
        st = solver.sync()
        if not math.isfinite(st["alpha"]):
            raise RuntimeError("non-finite wave speed after warm-up")
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(local)
        sampler.start()
        e0.record(stream)
        solver.advance_async(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        barrier(world)
        ms = e0.elapsed_time(e1)
        st = solver.sync()
        prof = solver.profile_steps(args.profile_steps) if args.profile_steps > 0 else None
        return solver, ms, st, clocks, prof

    primary = N.PREC_FP64 if args.precision == "fp64" else N.PREC_MIXED
    solver, ms, st, clocks, prof = timed(primary)
    ms_max = dist_max(ms, world)
    value = nt * 3 * args.steps * world / (ms_max / 1e3)

    # roofline of the dominant kernel (instrumented pass of the same kernels on the same stream)
    # measured DFMA throughput of this GPU: the roofline of the FP64 path
    try:
        fp64_meas, _ = N.probe_fma_peak(N.PREC_FP64)
    except Exception:
        fp64_meas = None
    roof = None
    if prof:
        kinds = {k: v for k, v in prof.items() if v[1] > 0}
        dom = max(kinds, key=lambda k: kinds[k][0])
        total_ms = sum(v[0] for v in kinds.values())
        avg_ms = kinds[dom][0] / kinds[dom][1]
        flops = ALGO_FLOPS_P2.get(dom, 0.0) * nt
        achieved = flops / (avg_ms / 1e3) / 1e12 if flops else None
        ex = EXECUTED_FLOPS_P2.get(dom)
        peak = fp64_meas if fp64_meas else FP64_PEAK_TFLOPS
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None,
                "traffic": TRAFFIC_PER_LAUNCH.get(dom),
                "peak_source": ("measured DFMA throughput (dg_probe_fma_peak, this run)" if fp64_meas else
                                "derived FP64 peak: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (of recipe nominal)"),
                "peak_measured": fp64_meas, "peak_derived": FP64_PEAK_TFLOPS,
                "frac_of_derived": achieved / FP64_PEAK_TFLOPS if achieved else None,
                "algorithmic_flops_per_cell": ALGO_FLOPS_P2.get(dom),
                "executed_flops_per_cell": ex,
                "executed_tflops": ex * nt / (avg_ms / 1e3) / 1e12 if ex else None,
                "avg_launch_ms": avg_ms,
                "kernel_share": {k: round(v[0] / total_ms, 4) for k, v in kinds.items()},
                "instrumented_ms_per_step": total_ms / args.profile_steps}

    # end-to-end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        ne = min(args.steps, 10)
        host = torch.empty(u0.shape, dtype=torch.float64, pin_memory=True).numpy()
        u, t = solver.get_state()
        host[...] = u
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(ne):
            solver.set_state(host, t)                 # H2D from pinned memory
            solver.advance(1e30, max_steps=1)
            _, t = solver.get_state(out=host)         # D2H into the same pinned buffer
        el = dist_max(time.perf_counter() - t0, world)
        nbytes = int(u0.size * 8)
        e2e = {"value": nt * 3 * ne * world / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": ne}

    # FP32 form (FP32 modes / flux arithmetic, FP64 averages and limiter)
    mixed = None
    if not args.no_mixed:
        try:
            s2, ms2, st2, clocks2, prof2 = timed(N.PREC_MIXED)
            ms2 = dist_max(ms2, world)
            mixed = {"value": nt * 3 * args.steps * world / (ms2 / 1e3), "ms_per_step": ms2 / args.steps,
                     "dtype": "f32+f64avg", "speedup_vs_fp64": ms / ms2}
            if prof2:
                k2 = {k: v for k, v in prof2.items() if v[1] > 0}
                tot2 = sum(v[0] for v in k2.values())
                mixed["kernel_share"] = {k: round(v[0] / tot2, 4) for k, v in k2.items()}
                # HBM roofline of each stage kernel of the mixed form on the
                # method's bytes, the dominant one as the line's roofline
                hbm = peaks.get("hbm_gbs", 6800.0)
                if wl.k == 2:
                    per = {}
                    for kk in ("rk", "stats", "oe_bp"):
                        if kk not in k2:
                            continue
                        avg_k = k2[kk][0] / k2[kk][1]
                        gbs = ALGO_BYTES_MIXED_P2[kk] * nt / (avg_k / 1e3) / 1e9
                        per[kk] = {"bound": "hbm", "kernel": kk, "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                   "frac": gbs / hbm, "traffic": TRAFFIC_MIXED_PER_LAUNCH.get(kk),
                                   "peak_source": f"{peak_src} HBM copy bandwidth",
                                   "algorithmic_bytes_per_cell": ALGO_BYTES_MIXED_P2[kk], "avg_launch_ms": avg_k}
                    dom2 = max(per, key=lambda kk: per[kk]["avg_launch_ms"])
                    mixed["roofline"] = per[dom2]
                    mixed["kernel_rooflines"] = per
                    mixed["step_hbm_frac"] = (sum(ALGO_BYTES_MIXED_P2.values()) * nt * 3 * args.steps
                                              / (ms2 / 1e3) / 1e9 / hbm)
            del s2
            # density L1 difference from the FP64 path after the same number of steps
            n_l1 = 20
            sa = N.Solver(mesh, N.config_for(wl, precision=N.PREC_MIXED), u0)
            sb = N.Solver(mesh, N.config_for(wl, precision=N.PREC_FP64), u0)
            sa.advance(1e30, max_steps=n_l1)
            sb.advance(1e30, max_steps=n_l1)
            ua, _ = sa.get_state()
            ub, _ = sb.get_state()
            area = mesh.geometry(wl.k)["area"]
            mixed["density_l1_rel_vs_fp64"] = float((np.abs(ua[0, 0] - ub[0, 0]) * area).sum()
                                                    / (np.abs(ub[0, 0]) * area).sum())
            mixed["density_l1_steps"] = n_l1
            del sa, sb
        except Exception as exc:      # mixed precision not available
            mixed = {"error": str(exc)}

    # batch of 64 independent solves over one work list, launch form and shape autotuned
    batch = None
    if not args.no_batch:
        from paper_2409_09620_gb300 import workloads as W
        wls = W.batch_workloads(64)
        bmeshes = [N.Mesh.from_mesh(w.mesh) for w in wls]
        bus = [N.initial_state(m, w) for m, w in zip(bmeshes, wls)]
        cells = sum(m.nt for m in bmeshes)
        batch = {"solves": len(wls), "cells": cells, "p2_solves": sum(w.k == 2 for w in wls),
                 "cells_min": min(m.nt for m in bmeshes), "cells_max": max(m.nt for m in bmeshes)}
        for label, prec in (("fp64", N.PREC_FP64), ("fp32", N.PREC_MIXED)):
            bt = N.Batch(bmeshes, [N.config_for(w, precision=prec) for w in wls], bus)
            tune = bt.autotune(steps=2)
            stream = torch.cuda.ExternalStream(bt.solver(0).stream)
            bt.advance_async(args.warmup)
            bt.sync()
            barrier(world)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bt.advance_async(args.batch_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            bt.sync()
            bms = dist_max(e0.elapsed_time(e1), world)
            batch[label] = {"value": cells * 3 * args.batch_steps * world / (bms / 1e3),
                            "ms_per_step": bms / args.batch_steps, "shape": bt.shape(), "autotune": tune}
            del bt

    # serving: Poisson arrivals of solve requests (cells log-uniform in
    # [1k, 500k], P1 / P2, vortex / blast / four-quadrant data, end times
    # U[0.05, 0.5]), continuous batching.  The same seeded requests arrive at
    # each rate of the sweep; aggregate throughput stops rising once the
    # device is saturated, and the latencies there are the reported ones.
    serving = None
    if not args.no_serving:
        from paper_2409_09620_gb300 import workloads as W

        def serve_run(n, rate, precision):
            reqs = W.serving_requests(n, rate=rate, cmin=1000, cmax=500000, t_end=(0.05, 0.5))
            payload = []
            for wl_r, te, at in reqs:
                m = N.Mesh.from_mesh(wl_r.mesh)
                payload.append((wl_r, N.config_for(wl_r, precision=precision), N.initial_state(m, wl_r), te, at))
                m.close()
            srv = N.Server(precision, budget_bytes=64 << 30, steps_per_tick=args.serve_steps_per_tick)
            barrier(world)
            t0 = time.perf_counter()
            ids, nxt, max_run = [], 0, 0
            while True:
                now = time.perf_counter() - t0
                while nxt < len(payload) and payload[nxt][4] <= now:
                    wl_r, cf_r, u_r, te, _ = payload[nxt]
                    ids.append(srv.submit(wl_r.mesh, cf_r, u_r, te))
                    nxt += 1
                r, q = srv.tick()
                max_run = max(max_run, r)
                if r == 0 and q == 0:
                    if nxt == len(payload):
                        break
                    time.sleep(max(0.0, payload[nxt][4] - (time.perf_counter() - t0)))
            makespan = dist_max(time.perf_counter() - t0, world)
            infos = [srv.info(i) for i in ids]
            srv.close()
            lat = np.array([f["done_s"] - f["submit_s"] for f in infos])
            done_cells = sum(f["cells"] * 3 * f["steps"] for f in infos)
            return {"requests": len(ids), "rate_per_s": rate,
                    "failed": int(sum(f["state"] != N.REQ_DONE for f in infos)),
                    "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                    "mean_latency_s": float(lat.mean()), "makespan_s": makespan,
                    "throughput": done_cells * world / makespan, "unit": UNIT, "max_running": max_run,
                    "cells_range": [int(min(f["cells"] for f in infos)), int(max(f["cells"] for f in infos))],
                    "cell_stages": int(done_cells), "steps_total": int(sum(f["steps"] for f in infos))}

        rates = [float(r) for r in args.serve_rates.split(",") if r]
        serving = {"config": "requests of 1k-500k cells (log-uniform), P1/P2, vortex / blast / four-quadrant "
                             "Riemann data, t_end U[0.05, 0.5], Poisson arrivals; 64 GiB budget, "
                             f"{args.serve_steps_per_tick} steps per tick",
                   "mixed": [serve_run(args.serve_requests, r, N.PREC_MIXED) for r in rates]}
        thr = [x["throughput"] for x in serving["mixed"]]
        best = int(np.argmax(thr))
        serving["mixed_saturating"] = {"rate_per_s": rates[best], "throughput": thr[best],
                                       "p50_latency_s": serving["mixed"][best]["p50_latency_s"],
                                       "p99_latency_s": serving["mixed"][best]["p99_latency_s"],
                                       "plateau": len(thr) > 1 and thr[-1] < 1.1 * thr[-2]}
        if args.serve_fp64_requests > 0:
            serving["fp64"] = serve_run(args.serve_fp64_requests, max(rates), N.PREC_FP64)

    # the paper's headline: optimal vs classical decomposition, steps and time to
    # the same end time (BP time step of Sec. 5 with either CFL number)
    cfl_gain = None
    if not args.no_cfl_gain:
        from paper_2409_09620_gb300 import workloads as W
        cfl_gain = {"workload": "dmr720x180 (259,200 cells), FP64, RIOE + BP, to t = T"}
        for k, T in ((1, 1e-3), (2, 1e-3)):
            wl_g = W.dmr_workload(nx=720, ny=180, k=k)
            m_g = N.Mesh.from_mesh(wl_g.mesh)
            u_g = N.initial_state(m_g, wl_g)
            res = {}
            for name, dc in (("optimal", 0), ("classical", 1)):
                sv = N.Solver(m_g, N.config_for(wl_g, decomp=dc), u_g)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st_g, _ = sv.advance(T)
                el = time.perf_counter() - t0
                res[name] = {"steps": st_g["steps"], "seconds": el, "mean_dt": T / st_g["steps"]}
                del sv
            cfl_gain[f"P{k}"] = {"T": T, **{n: v for n, v in res.items()},
                                 "mean_dt_ratio": res["classical"]["steps"] / res["optimal"]["steps"],
                                 "time_ratio": res["classical"]["seconds"] / res["optimal"]["seconds"],
                                 "min_cfl_area_ratio": m_g.min_cfl_area(k, 0) / m_g.min_cfl_area(k, 1)}
        cfl_gain["paper_dmr_mean_dt_ratio"] = {"P1": 2.869570, "P2": 4.486689}

    # the problem to an end time: steps, counters (limited cells, cell averages
    # outside G at any stage, CFL breaches), wall time, the smallest density,
    # and the density L1 difference of the mixed form from FP64
    to_t_end = None
    if args.to_t_end > 0.0 and args.workload == "dmr":
        from paper_2409_09620_gb300 import workloads as W

        def run_to_end(m, w, u, prec, T):
            sv = N.Solver(m, N.config_for(w, precision=prec), u)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st_e, rc_e = sv.advance(T, check=False)
            el = time.perf_counter() - t0
            ue = sv.get_state()[0]
            del sv
            return ue, {"steps": st_e["steps"], "t": st_e["t"], "status": rc_e, "seconds": el,
                        "limited_cells": st_e["limited_cells"], "nonphysical": st_e["nonphysical"],
                        "cfl_breaches": st_e["cfl_breaches"], "alpha_last": st_e["alpha"],
                        "density_min": float(ue[0, 0].min()),
                        "cell_stages_per_s": m.nt * 3 * st_e["steps"] / el}

        def density_l1(m, w, a, b):
            area = m.geometry(w.k)["area"]
            return float((np.abs(a[0, 0] - b[0, 0]) * area).sum() / (np.abs(b[0, 0]) * area).sum())

        T = args.to_t_end
        to_t_end = {"t_end": T}
        gx, gy = (int(v) for v in args.to_t_end_grid.split("x"))
        w_r = W.dmr_workload(nx=gx, ny=gy, k=2)
        m_r = N.Mesh.from_mesh(w_r.mesh)
        u_r = N.initial_state(m_r, w_r)
        ua, ra = run_to_end(m_r, w_r, u_r, N.PREC_MIXED, T)
        ub, rb = run_to_end(m_r, w_r, u_r, N.PREC_FP64, T)
        to_t_end[f"dmr{gx}x{gy}"] = {"cells": w_r.mesh.nt, "mixed": ra, "fp64": rb,
                                     "density_l1_rel_mixed_vs_fp64": density_l1(m_r, w_r, ua, ub),
                                     "speedup_mixed_vs_fp64": rb["seconds"] / ra["seconds"]}
        del m_r
        # the reduced grid with a transmissive right side (the cell average as
        # its exterior state) instead of the pre-shock state there
        w_t = W.dmr_workload(nx=gx, ny=gy, k=2, right=W.BC_TRANSMISSIVE)
        m_t = N.Mesh.from_mesh(w_t.mesh)
        _, rt = run_to_end(m_t, w_t, N.initial_state(m_t, w_t), N.PREC_MIXED, T)
        to_t_end[f"dmr{gx}x{gy}_transmissive_right"] = {"cells": w_t.mesh.nt, "mixed": rt}
        del m_t
        uf, rf = run_to_end(mesh, wl, u0, N.PREC_MIXED, T)
        full = {"cells": nt, "mixed": rf}
        if args.to_t_end_transmissive:
            w_f = W.dmr_workload(nx=args.nx, ny=args.ny, k=2, right=W.BC_TRANSMISSIVE)
            m_f = N.Mesh.from_mesh(w_f.mesh)
            _, rft = run_to_end(m_f, w_f, N.initial_state(m_f, w_f), N.PREC_MIXED, T)
            to_t_end[f"{args.workload}{args.nx}x{args.ny}_transmissive_right"] = {"cells": w_f.mesh.nt, "mixed": rft}
            del m_f
        if args.to_t_end_full_fp64:
            ug, rg = run_to_end(mesh, wl, u0, N.PREC_FP64, T)
            full["fp64"] = rg
            full["density_l1_rel_mixed_vs_fp64"] = density_l1(mesh, wl, uf, ug)
            full["speedup_mixed_vs_fp64"] = rg["seconds"] / rf["seconds"]
        to_t_end[f"{args.workload}{args.nx}x{args.ny}"] = full
        del uf

    sedov = None
    if args.sedov_t_end > 0.0:
        from paper_2409_09620_gb300 import workloads as W
        w_s = W.sedov_workload(n=256, k=2)
        m_s = N.Mesh.from_mesh(w_s.mesh)
        sv = N.Solver(m_s, N.config_for(w_s), N.initial_state(m_s, w_s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st_s, rc_s = sv.advance(args.sedov_t_end, check=False)
        el = time.perf_counter() - t0
        us_, _ = sv.get_state()
        area = m_s.geometry(2)["area"]
        sedov = {"workload": "sedov256x256_P2 (131,072 cells), FP64", "t_end": args.sedov_t_end,
                 "steps": st_s["steps"], "t": st_s["t"], "status": rc_s, "seconds": el,
                 "limited_cells": st_s["limited_cells"], "nonphysical": st_s["nonphysical"],
                 "cfl_breaches": st_s["cfl_breaches"], "density_min": float(us_[0, 0].min()),
                 "density_max": float(us_[0, 0].max()),
                 "mass": float((us_[0, 0] * area).sum()), "energy": float((us_[3, 0] * area).sum()),
                 "cell_stages_per_s": m_s.nt * 3 * st_s["steps"] / el}
        del sv, m_s

    # the paper's own domains (Sec. 5) on near-equilateral lattice meshes of
    # about its cell counts: throughput, and the mean BP time step of the
    # optimal over the classical decomposition over the first steps
    paper_meshes = None
    if not args.no_paper_meshes:
        from paper_2409_09620_gb300 import workloads as W

        def ms_per_step(m, w, u, precision, n):
            sv = N.Solver(m, N.config_for(w, precision=precision), u)
            stream = torch.cuda.ExternalStream(sv.stream)
            sv.advance_async(3)
            sv.sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sv.advance_async(n)
            e1.record(stream)
            sv.sync()
            return e0.elapsed_time(e1) / n

        paper_meshes = {}
        for key, make, paper in (
                ("ffs", lambda k: W.ffs_workload(k=k),
                 {"cells": 73862, "mean_dt_ratio": {"P1": 2.851852, "P2": 4.489796}}),
                ("wedge_dmr", lambda k: W.wedge_dmr_workload(k=k),
                 {"cells": 828840, "mean_dt_ratio": {"P1": 2.869570, "P2": 4.486689}})):
            ent = {"paper": paper}
            for k in (1, 2):
                w = make(k)
                m = N.Mesh.from_mesh(w.mesh)
                u = N.initial_state(m, w)
                ent["cells"] = w.mesh.nt
                if k == 2:
                    for pname, prec in (("fp64", N.PREC_FP64), ("mixed", N.PREC_MIXED)):
                        ms_k = ms_per_step(m, w, u, prec, 20)
                        ent[f"P2_{pname}"] = {"ms_per_step": ms_k, "value": w.mesh.nt * 3 / (ms_k / 1e3),
                                              "unit": UNIT}
                # 30 steps of the optimal decomposition set the end time; the
                # classical one runs to the same time
                s_opt = N.Solver(m, N.config_for(w, decomp=0), u)
                a_st, _ = s_opt.advance(10.0, max_steps=30)
                T = a_st["t"]
                s_zxs = N.Solver(m, N.config_for(w, decomp=1), u)
                b_st, _ = s_zxs.advance(T)
                ent[f"P{k}_dt"] = {"T": T, "optimal_steps": a_st["steps"], "classical_steps": b_st["steps"],
                                   "mean_dt_ratio": b_st["steps"] / a_st["steps"],
                                   "min_cfl_area_ratio": m.min_cfl_area(k, 0) / m.min_cfl_area(k, 1)}
                del s_opt, s_zxs
            paper_meshes[key] = ent

    # scalar conservation laws (Sec. 2, Sec. 5 accuracy studies): errors and
    # orders on a mesh and its refinements, and throughput on the finest mesh
    scalar = None
    if not args.no_scalar:
        from paper_2409_09620_gb300 import workloads as W
        paper_l1 = {  # the paper's tables tab:Ex_LinearS1 and tab:Ex_BurgS1, N = 176 * 4^i
            "linear": {"P1": [8.18e-2, 1.56e-2, 2.79e-3, 4.76e-4, 9.11e-5, 2.01e-5],
                       "P2": [5.29e-2, 2.90e-3, 9.15e-5, 5.70e-6, 4.85e-7, 5.10e-8],
                       "P3": [4.45e-2, 3.20e-4, 3.01e-6, 8.89e-8, 3.08e-9, 1.23e-10]},
            "burgers": {"P1": [1.88e-2, 3.77e-3, 7.57e-4, 1.68e-4, 4.10e-5, 1.02e-5],
                        "P2": [3.05e-3, 3.22e-4, 3.52e-5, 3.95e-6, 4.82e-7, 6.28e-8],
                        "P3": [1.20e-3, 3.39e-5, 1.28e-6, 6.11e-8, 2.97e-9, 1.58e-10]}}
        scalar = {"mesh": "periodic jittered 5x5 grid refined L times by quadrisection (50 * 4^L cells)",
                  "time": "SSP-RK(2,2) for P1, SSP-RK(3,3) for P2 and P3; P3 dt scaled by (h/h_1)^(1/3)",
                  "paper_L1": paper_l1, "paper_cells": [176, 704, 2816, 11264, 45056, 180224]}
        levels = range(1, 6)
        for name, make in (("linear", W.scalar_linear_workload), ("burgers", W.scalar_burgers_workload)):
            tab = {}
            for k in (1, 2, 3):
                rows, prev = [], None
                for lev in levels:
                    wl_s = make(level=lev, k=k)
                    m = N.Mesh.from_mesh(wl_s.mesh)
                    u = N.scalar_project(m, k, wl_s.u0)
                    cf = N.make_scalar_config(k, flux=wl_s.flux, cfl=0.5 ** ((lev - 1) / 3.0) if k == 3 else 1.0)
                    sv = N.ScalarSolver(m, cf, u)
                    st_s = sv.advance(wl_s.t_end)
                    xy = m.quad_points()
                    e = np.array(sv.errors(wl_s.exact(xy[..., 0], xy[..., 1], wl_s.t_end)))
                    row = {"cells": wl_s.mesh.nt, "steps": st_s["steps"], "L1": e[0], "L2": e[1], "Linf": e[2]}
                    if prev is not None:
                        row["order"] = [float(v) for v in np.log2(prev / e)]
                    rows.append(row)
                    prev = e
                    sv.close()
                tab[f"P{k}"] = rows
            scalar[name] = tab
        thr = {}
        wl6 = W.scalar_linear_workload(level=6, k=1)
        m6 = N.Mesh.from_mesh(wl6.mesh)
        for k in (1, 2, 3):
            sv = N.ScalarSolver(m6, N.make_scalar_config(k, flux=1), N.scalar_project(m6, k, W.burgers_smooth))
            stream = torch.cuda.ExternalStream(sv.stream)
            sv.advance_async(5)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sv.advance_async(50)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_s = e0.elapsed_time(e1) / 50
            stages = 2 if k == 1 else 3
            thr[f"P{k}"] = {"ms_per_step": ms_s, "value": wl6.mesh.nt * stages / (ms_s / 1e3), "unit": UNIT,
                            "cells": wl6.mesh.nt, "flux": "burgers"}
            sv.close()
        scalar["throughput"] = thr

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(make_workload(args.workload, args.nx, args.ny))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded jittered grid, analytic initial state)",
                "config": {"workload": f"{args.workload}{args.nx}x{args.ny}_P2" if args.workload != "vortex"
                           else f"vortex{args.nx}_P1", "cells": nt, "k": wl.k, "precision": "fp64",
                           "oe": "RI", "bp": "optimal-points", "cfl": 1.0,
                           "l2": "working set ~1.7 GB > 129 MB L2, no flush"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": 19 * args.steps, "clocks": clocks, "fp32": mixed, "batch": batch,
                "serving": serving, "bp_cfl_gain": cfl_gain, "paper_meshes": paper_meshes, "scalar": scalar,
                "to_t_end": to_t_end, "sedov_to_t_end": sedov,
                "peaks": {"source": peak_src, "hbm_gbs": peaks.get("hbm_gbs")},
                "stats": {"limited_cells": st["limited_cells"], "nonphysical": st["nonphysical"],
                          "cfl_breaches": st["cfl_breaches"],
                          "t": st["t"], "dt_last": st["dt_last"]}}
        print(json.dumps(line), flush=True)
    barrier(world)


if __name__ == "__main__":
    main()
