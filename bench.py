#!/usr/bin/env python3
"""Throughput of the MGEnKF analysis cycle on one GB300 (or N).

Default workload: 96 independent 2-D Navier-Stokes assimilation problems
(coarse grids 64^2..192^2, fine grids 4x per side, 16..128 members,
256..2048 observations each), the largest single-GPU configuration.  One
"step" is one analysis cycle of every problem (Algorithm 4): forecast of each
fine run and all members over 10 model steps, the coarse-mesh EnKF analysis,
the prolonged correction of the fine run, one CUDA graph launch.  Mixed
precision: FP32 states and forecasts, BF16 anomaly products with FP32
accumulation, FP64 means, covariances and Cholesky.  `value` = problem-cycles
per second over all ranks (the 96 problems are sharded over the ranks, no
collective on the data path).  Other workloads (--workload): burgers_large
(fine 16384 / coarse 4096, Ne = 128), ns2d (512^2 / 128^2, Ne = 64), ns2d_cnn
(learned correction, 1024^2 / 256^2), dual (Dual EnKF on the Burgers inlet).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on this host's cores on bounded samples of the same workload.
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


# Per workload: algorithmic FP32 flops per point-step of the forecast, the
# forecast kernel timed for the roofline, its launches per model step, the
# DRAM bytes per launch measured by ncu for the current kernel (None when not
# captured), and the precision of the synthetic truth run.
WORKLOADS = {
    # SSP-RK3 Burgers, k-form in the scaled variable v = a u, dt L from edge
    # differences shared by neighbouring points: 3 x 7 (dt L) + 1 + 3 + 4
    # (stages) + 3 (Fast2Sum) = 32 flops (an FMA counts 2); as FP32 operations
    # (FADD, FMUL, FFMA one each): 3 x 6 (dt L) + 1 + 2 + 5 (stages, the last
    # with the Fast2Sum compensation) = 26
    # The forecast is two launches of the kernel that run side by side (the fine
    # run on its own cluster, the members after it by programmatic
    # serialisation); the roofline takes them as one unit, and traffic is the sum
    # of the two launches' DRAM bytes
    "burgers_large": dict(flops=32, bytes=8, kernel="burgers_f32x2_kernel<4> fine run + <8> members",
                          launches_per_step=None, traffic=2410752, truth="fp32"),
    # NS-2D, one model step (three RK stages fused in one launch): algorithmic
    # FP32 flops per point-step counted from the kernels' arithmetic (an FMA
    # counts 2, the halo recomputation is not counted): per stage 114 for dt L
    # (nodal inviscid fluxes 20, their differences 16, three face fluxes of 21
    # each, the face differences 15: each face is counted once) and 11 for the
    # primitives of its input, plus 8 + 20 + 20 for the three stage updates:
    # 3 x 125 + 48 = 423.  Algorithmic bytes: the state read and
    # written once per step, 2 x 4 variables x 4 B = 32 per point-step.
    # The handle's forecast is the column march (autotuned layout), the members
    # and the fine run on two streams: one launch each per model step, side by
    # side; the roofline takes the whole forecast as one unit.
    "ns2d": dict(flops=423, bytes=32, kernel="ns2d_rk3_march<TableUnits> members + fine run",
                 launches_per_step=None, traffic=None, truth="fp64"),
    # NS-2D 1024^2 / 256^2 with the learned correction of the prolongation
    "ns2d_cnn": dict(flops=423, bytes=32, kernel="ns2d_rk3_march<TableUnits> members + fine run",
                     launches_per_step=None, traffic=None, truth="fp64"),
    # Dual EnKF parameter estimation on the Burgers inlet model (latency-bound: small grids)
    "dual": dict(kernel="k_burgers_inlet"),
    # 96 independent NS-2D problems: one march launch per model step and grid
    # size.  traffic_per_point_step: dram__bytes_read.sum + dram__bytes_write.sum
    # per point-step of the march launches of one cycle, measured by ncu on the
    # 8-problem batch (16.71 B read, 4.45 B written: ncu counts the lines L2
    # evicts during a launch; two-part cycle, autotuned choices), scaled to this
    # batch by its point-steps; None once the kernel changes.
    "batched": dict(flops=423, bytes=32, kernel="ns2d_rk3_march<TableUnits>", launches_per_step=None,
                    traffic_per_point_step=21.15, truth="fp32"),
}
CNN_FLOPS_PER_PIXEL = 2 * 9 * (8 * 32 + 32 * 32 + 32 * 64)  # three 3x3 convolutions per coarse pixel


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--fp64-cycles", type=int, default=40,
                    help="cycles of the plain FP64 run compared at equal RMSE")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="batched",
                    help="batched (default: 96 independent NS-2D problems of uneven sizes, one graph launch per "
                         "cycle), burgers_large (fine 16384 / coarse 4096, Ne=128), ns2d "
                         "(fine 512^2 / coarse 128^2, Ne=64, 2048 observations), ns2d_cnn "
                         "(fine 1024^2 / coarse 256^2, Ne=64, learned prolongation correction) or "
                         "dual (inlet-parameter estimation on the Burgers inlet model, 800 nodes, ratio 4)")
    ap.add_argument("--cnn-pairs", type=int, default=2000,
                    help="training pairs generated for ns2d_cnn (cycles of lockstep runs; 2000 take "
                         "about 90 s to generate on one GB300)")
    ap.add_argument("--cnn-epochs", type=int, default=10)
    ap.add_argument("--tiles", default=None,
                    help="batched: JSON tile table to load (autotuned and written there if missing)")
    ap.add_argument("--problems", type=int, default=96, help="batched: number of problems")
    ap.add_argument("--forecast-choice", default="auto",
                    help="ns2d, ns2d_cnn: layout of the handle's forecast, 'auto' (autotuned) or two "
                         "choices 'members,fine' (see mgenkf_set_forecast_choice; -1,-1 the tile kernel)")
    ap.add_argument("--filter", type=float, default=None,
                    help="ns2d: add an ablation of the centred sixth-order filter of the NS model "
                         "(this strength after every model step): cycles/s and RMSE against no filter")
    ap.add_argument("--recentre", action="store_true",
                    help="burgers_large / ns2d: add an ablation of the fine-to-coarse feedback "
                         "(ensemble re-centred on the restricted fine forecast)")
    ap.add_argument("--regularise", type=float, default=None,
                    help="burgers_large / ns2d: final fine iteration (Algorithm 4 step 6) with this "
                         "relaxation in the timed cycles, plus an alpha = 0 / alpha ablation")
    return ap.parse_args()


# --------------------------------------------------------------------------
# distributed plumbing (host side only: barrier and max of the timings)
# --------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except (OSError, ValueError):
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def measure_alu_peaks(M, torch, stream):
    """FP32 and FP64 FMA-pipe throughput on this GPU, measured with the
    library's probe kernel (eight independent FMA chains per thread, four CTAs
    of 256 threads per SM), best of three launches of about 5 ms each, CUDA
    events on `stream`."""
    out = {}
    n = M.mgk_fma_probe_threads()
    for name, fp64, iters, dt in (("fp32", 0, 160000, torch.float32), ("fp64", 1, 2600, torch.float64)):
        sink = torch.empty(n, dtype=dt, device="cuda")
        with torch.cuda.stream(stream):
            M.mgk_fma_probe(fp64, iters, sink, stream=stream.cuda_stream)  # warm-up
            best = 0.0
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                flops = M.mgk_fma_probe(fp64, iters, sink, stream=stream.cuda_stream)
                b.record(stream)
                b.synchronize()
                best = max(best, flops / (a.elapsed_time(b) / 1e3))
        out[f"{name}_tflops"] = best / 1e12
    out["how"] = ("mgk_fma_probe: 8 independent FMA chains per thread, 4 x 256 threads per SM, "
                  "best of 3 launches (CUDA events); an FMA counts 2 flops")
    return out


# --------------------------------------------------------------------------
# reference arm and CPU baseline: the FP64 oracle on this host's cores
# --------------------------------------------------------------------------
def oracle_cycle_sample(w, inp, mg, step_fraction: int):
    """Time one bounded sample of a cycle: 1/step_fraction of the forecast
    steps plus one full analysis, prolongation and RMSE; returns the time
    scaled to a full cycle."""
    import oracle as O
    steps = max(1, w.steps_per_cycle // step_fraction)
    t0 = time.perf_counter()
    mg.forecast(steps)
    t1 = time.perf_counter()
    from paper_2012_10091_gb300 import workloads as W
    yo = W.sample_truth(w, inp["truth0"], inp["obs_idx"], inp["obs_var"])
    mg.analyse(yo)
    mg.prolong_correct()
    O.rmse(mg.fine, inp["truth0"], w.V)
    t2 = time.perf_counter()
    return (t1 - t0) * (w.steps_per_cycle / steps) + (t2 - t1)


def cpu_threads():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def cpu_baseline(w, inp):
    import oracle as O
    mg = O.MGEnKF(w.model, w.nf, w.ratio, w.length, w.dt, inp["fine0"], inp["members0"],
                  inp["obs_idx"], inp["obs_var"], w.sigma, w.seed, nu=w.nu)
    t = oracle_cycle_sample(w, inp, mg, 1)
    # the same oracle on one core: 1/16 of the forecast steps (time scaled by
    # 16) plus one full analysis, prolongation and RMSE
    try:
        O.set_threads(1)
        t1 = oracle_cycle_sample(w, inp, mg, 16)
    finally:
        O.set_threads(cpu_threads())
    return {"value": 1.0 / t, "unit": "cycles/s", "cores": cpu_threads(), "kind": "oracle",
            "sample": f"1 full cycle of {w.name} ({w.steps_per_cycle} RK3 steps of the fine run and "
                      f"{w.ne} members, ensemble-space FP64 analysis, prolongation, RMSE), "
                      f"OpenMP over members, {cpu_threads()} threads",
            "single_thread": {"value": 1.0 / t1, "unit": "cycles/s", "cores": 1,
                              "sample": f"{w.steps_per_cycle // 16} of the {w.steps_per_cycle} forecast "
                                        f"steps (time scaled by 16) plus one full analysis, "
                                        f"prolongation and RMSE, 1 thread"}}


def run_reference(args, dist, w, inp):
    if dist.rank != 0:
        return
    import oracle as O
    O.build()
    frac = 32
    mg = O.MGEnKF(w.model, w.nf, w.ratio, w.length, w.dt, inp["fine0"], inp["members0"],
                  inp["obs_idx"], inp["obs_var"], w.sigma, w.seed, nu=w.nu)
    for _ in range(args.warmup):
        oracle_cycle_sample(w, inp, mg, frac)
    times = [oracle_cycle_sample(w, inp, mg, frac) for _ in range(args.steps)]
    per = float(np.mean(times))
    val = 1.0 / per
    sample = (f"per step: {w.steps_per_cycle // frac} of the {w.steps_per_cycle} RK3 steps of a "
              f"cycle (time scaled by {frac}) plus one full FP64 analysis, prolongation and RMSE")
    line = {"metric": METRIC[args.workload],
            "value": val, "unit": "cycles/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w.name, "nf": w.nf, "nc": w.nc, "ne": w.ne, "ny": w.ny,
                       "steps_per_cycle": w.steps_per_cycle, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": "cycles/s", "kind": "oracle",
                             "cores": cpu_threads(), "sample": sample},
            "e2e": {"value": val, "unit": "cycles/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def truth_and_obs(M, w, inp, ncycles, torch, truth_prec):
    """Synthetic input: truth trajectory on the GPU and its noisy samples at
    the observed nodes, one row per cycle (resident in HBM)."""
    fp32 = truth_prec == "fp32"
    truth = torch.tensor(inp["truth0"], dtype=torch.float32 if fp32 else torch.float64, device="cuda")
    truths = torch.empty((ncycles, w.nxf), dtype=torch.float64, device="cuda")
    yos = torch.empty((ncycles, w.ny), dtype=torch.float64, device="cuda")
    nfp = w.nf ** w.dim
    idx = torch.tensor(inp["obs_var"].astype(np.int64) * nfp + inp["obs_idx"], device="cuda")
    model = M.MGENKF_BURGERS1D if w.model == "burgers1d" else M.MGENKF_NS2D
    for k in range(ncycles):
        M.mgk_forecast(model, M.MGENKF_MIXED if fp32 else M.MGENKF_FP64, truth, 1, w.nf, w.length,
                       w.dt, w.nu, w.gamma, w.prandtl, nsteps=w.steps_per_cycle,
                       stream=torch.cuda.current_stream().cuda_stream)
        truths[k] = truth.double()
        from paper_2012_10091_gb300 import workloads as W
        yos[k] = truths[k][idx] + torch.tensor(W.observation_noise(w, k), device="cuda")
    torch.cuda.synchronize()
    return truths, yos


def _forecast_choice(g, args):
    """Autotune the handle's forecast layout, or set the one given (NS-2D
    workloads; the Burgers forecast has no layout to choose)."""
    if getattr(args, "workload", "ns2d") not in ("ns2d", "ns2d_cnn"):
        return g.forecast_choice()
    if args.forecast_choice == "auto":
        return g.forecast_autotune(reps=3)
    m, f = (int(x) for x in args.forecast_choice.split(","))
    g.set_forecast_choice(m, f)
    return g.forecast_choice()


def _layout(M, choice):
    """Column-march layout of a handle's forecast (members, fine run) for the
    config: rows per segment and narrow bands per grid."""
    if choice[0] < 0:
        return "2-D tile kernel, both grids in one launch per step"
    return {grid: {"segment_rows": M.SEGMENT_ROWS[c], "narrow_bands": M.NARROW_BANDS[c]}
            for grid, c in zip(("members", "fine"), choice)}


def run_gpu(args, dist, w, inp):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_10091_gb300 import mgenkf as M

    dev = dist.local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    ncyc = args.warmup + args.steps
    spec = WORKLOADS[args.workload]
    with torch.cuda.stream(stream):
        truths, yos = truth_and_obs(M, w, inp, max(ncyc, args.fp64_cycles, 10 if args.regularise else 0),
                                    torch, spec["truth"])
    torch.cuda.synchronize()

    g = M.MGEnKF.from_workload(w, stream=sp)
    g.set_state(inp["fine0"], inp["members0"])
    fc_choice = _forecast_choice(g, args)  # NS-2D: the march layout per grid; Burgers: nothing to choose
    if args.regularise is not None:
        g.set_regularisation(args.regularise)
    rmse_dev = torch.zeros((ncyc, w.V), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            M.mgenkf_cycle(g.h, w.steps_per_cycle, yos[k], truths[k], rmse_dev[k])
    torch.cuda.synchronize()
    assert g.sync() == 0

    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    launches0 = M.mgk_kernel_launches()
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")
    with torch.cuda.stream(stream):
        for j in range(args.steps):
            k = args.warmup + j
            flush.fill_(float(j))                      # evict L2 between timed cycles
            e0, e1, e2 = ev[j]
            e0.record(stream)
            M.mgenkf_forecast(g.h, w.steps_per_cycle)
            e1.record(stream)
            M.mgenkf_analyse(g.h, yos[k])
            M.mgenkf_prolong_correct(g.h)
            M.mgenkf_rmse(g.h, truths[k], rmse_dev[k])
            e2.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - wall0
    launches = M.mgk_kernel_launches() - launches0
    dist.barrier()
    clk = clocks.stop()
    assert g.sync() == 0
    cyc_ms = [a.elapsed_time(c) for a, _, c in ev]
    fc_ms = [a.elapsed_time(b) for a, b, _ in ev]
    t_total = sum(cyc_ms) / 1e3
    t_max = dist.max(t_total)
    cycles_all = dist.sum(float(args.steps))
    value = cycles_all / t_max
    fc_mean = float(np.mean(fc_ms)) / 1e3
    rmse_mixed = rmse_dev[:, 0].cpu().numpy()

    # plain FP64 MGEnKF on the same GPU and inputs, first fp64_cycles cycles
    nref = args.fp64_cycles
    fp64_plain = None
    if nref > 0:
        g64 = M.MGEnKF.from_workload(w, precision="fp64", stream=sp)
        g64.set_state(inp["fine0"], inp["members0"])
        gm = M.MGEnKF.from_workload(w, stream=sp)
        gm.set_state(inp["fine0"], inp["members0"])
        r64 = torch.zeros((nref, w.V), dtype=torch.float64, device="cuda")
        rmx = torch.zeros((nref, w.V), dtype=torch.float64, device="cuda")
        e64a, e64b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e64a.record(stream)
            for k in range(nref):
                M.mgenkf_cycle(g64.h, w.steps_per_cycle, yos[k], truths[k], r64[k])
            e64b.record(stream)
            for k in range(nref):
                M.mgenkf_cycle(gm.h, w.steps_per_cycle, yos[k], truths[k], rmx[k])
        torch.cuda.synchronize()
        assert g64.sync() == 0 and gm.sync() == 0
        fp64_cps = nref / (e64a.elapsed_time(e64b) / 1e3)
        f64, m64 = g64.get_state()
        fmx, mmx = gm.get_state()
        half = slice(nref // 2, nref)
        rm64 = float(r64[half, 0].mean())
        rmmx = float(rmx[half, 0].mean())
        state_rel = float(np.max(np.abs(fmx - f64)) / np.max(np.abs(f64)))
        g64.close()
        gm.close()
        fp64_plain = {"cycles_per_s": fp64_cps, "cycles": nref,
                      "rmse_last_half": rm64, "mixed_rmse_last_half": rmmx,
                      "rmse_rel_diff": abs(rmmx - rm64) / rm64,
                      "fine_state_rel_diff": state_rel,
                      "speedup_mixed_vs_fp64": value / dist.world / fp64_cps}

    # final fine iteration, on the same inputs: (a) alpha = 0 throughout
    # (recorded, no sweep); (b) alpha = 0, then alpha on the last cycle only:
    # the sweep's effect on the conservativity residual of one analysed state;
    # (c) alpha throughout: its effect on the RMSE over the last half
    regularisation = None
    if args.regularise is not None and args.regularise > 0:
        nab = min(max(args.fp64_cycles, 10), truths.shape[0])
        comp = 0 if w.V == 1 else 2          # u (Burgers), rho v (NS: the paper's indicator)
        res = {}
        for tag, alphas in (("a", [0.0] * nab), ("b", [0.0] * (nab - 1) + [args.regularise]),
                            ("c", [args.regularise] * nab)):
            ga = M.MGEnKF.from_workload(w, stream=sp)
            ga.set_state(inp["fine0"], inp["members0"])
            ra = torch.zeros((nab, w.V), dtype=torch.float64, device="cuda")
            with torch.cuda.stream(stream):
                for k in range(nab):
                    ga.set_regularisation(alphas[k])
                    M.mgenkf_cycle(ga.h, w.steps_per_cycle, yos[k], truths[k], ra[k])
            torch.cuda.synchronize()
            assert ga.sync() == 0
            gres = ga.gamma_residual().reshape(w.V, -1)
            res[tag] = (float(np.sqrt(np.mean(gres[comp] ** 2))), float(ra[nab // 2:, 0].mean()))
            ga.close()
        regularisation = {"alpha": args.regularise, "cycles": nab,
                          "gamma_component": "u" if w.V == 1 else "rho v",
                          "gamma_rms_before_sweep": res["a"][0], "gamma_rms_after_sweep": res["b"][0],
                          "gamma_ratio_one_sweep": res["b"][0] / res["a"][0],
                          "rmse_last_half_alpha0": res["a"][1], "rmse_last_half": res["c"][1]}

    # fine-to-coarse feedback: RMSE over the last half with and without
    feedback = None
    if args.recentre:
        nab = min(max(args.fp64_cycles, 10), truths.shape[0])
        rm = {}
        for on in (False, True):
            ga = M.MGEnKF.from_workload(w, stream=sp)
            ga.set_state(inp["fine0"], inp["members0"])
            ga.set_recentre(on)
            ra = torch.zeros((nab, w.V), dtype=torch.float64, device="cuda")
            with torch.cuda.stream(stream):
                for k in range(nab):
                    M.mgenkf_cycle(ga.h, w.steps_per_cycle, yos[k], truths[k], ra[k])
            torch.cuda.synchronize()
            assert ga.sync() == 0
            rm[on] = ra[nab // 2:].mean(dim=0).cpu().numpy().tolist()
            ga.close()
        feedback = {"cycles": nab, "rmse_last_half_off": rm[False], "rmse_last_half_on": rm[True]}

    # sixth-order filter of the NS model: cost and RMSE over the last half with and without
    filt = None
    if args.filter is not None and w.V == 4:
        nab = min(max(args.fp64_cycles, 10), truths.shape[0])
        rm, cps = {}, {}
        for sg in (0.0, args.filter):
            ga = M.MGEnKF.from_workload(w, stream=sp)
            ga.set_state(inp["fine0"], inp["members0"])
            ga.set_filter(sg)
            ra = torch.zeros((nab, w.V), dtype=torch.float64, device="cuda")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                M.mgenkf_cycle(ga.h, w.steps_per_cycle, yos[0], truths[0], ra[0])   # warm-up
                e0.record(stream)
                for k in range(1, nab):
                    M.mgenkf_cycle(ga.h, w.steps_per_cycle, yos[k], truths[k], ra[k])
                e1.record(stream)
            torch.cuda.synchronize()
            assert ga.sync() == 0
            cps[sg] = (nab - 1) / (e0.elapsed_time(e1) / 1e3)
            rm[sg] = ra[nab // 2:].mean(dim=0).cpu().numpy().tolist()
            ga.close()
        filt = {"sigma": args.filter, "cycles": nab, "cycles_per_s_off": cps[0.0],
                "cycles_per_s_on": cps[args.filter], "rmse_last_half_off": rm[0.0],
                "rmse_last_half_on": rm[args.filter],
                "note": "mgenkf_cycle on device buffers, CUDA events; the truth run is unfiltered"}

    # e2e: the same cycle through the C ABI with host buffers (pinned), copies inside
    e2e = None
    if not args.no_e2e:
        ge = M.MGEnKF.from_workload(w, stream=sp)
        ge.set_state(inp["fine0"], inp["members0"])
        if fc_choice[0] >= 0:
            ge.set_forecast_choice(*fc_choice)
        if args.regularise is not None:
            ge.set_regularisation(args.regularise)
        y_h = torch.empty((ncyc, w.ny), dtype=torch.float64, pin_memory=True)
        y_h.copy_(yos[:ncyc].cpu())
        t_h = torch.empty((ncyc, w.nxf), dtype=torch.float64, pin_memory=True)
        t_h.copy_(truths[:ncyc].cpu())
        out_h = torch.empty((ncyc, w.V), dtype=torch.float64, pin_memory=True)
        for k in range(args.warmup):
            M.mgenkf_cycle(ge.h, w.steps_per_cycle, y_h[k], t_h[k], out_h[k])
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        for j in range(args.steps):
            k = args.warmup + j
            M.mgenkf_cycle(ge.h, w.steps_per_cycle, y_h[k], t_h[k], out_h[k])  # returns after D2H
        torch.cuda.synchronize()
        te = dist.max(time.perf_counter() - t0)
        ge.close()
        e2e = {"value": cycles_all / te, "unit": "cycles/s",
               "h2d_bytes_per_step": 8 * (w.ny + w.nxf), "d2h_bytes_per_step": 8 * w.V}

    # roofline of the dominant kernel (the forecast): algorithmic FP32 flops
    # per launch (an FMA counts 2; counted from the scheme without the halo
    # recomputation) over the launch's time, against the FP32 FMA throughput
    # measured on this GPU by the probe kernel; the HBM view (algorithmic bytes,
    # the state read and written once per launch) beside it
    peaks, peak_src = measured_peaks()
    alu = measure_alu_peaks(M, torch, stream)
    pts = w.ne * w.nc ** w.dim + w.nf ** w.dim
    lps = spec["launches_per_step"]
    launches_fc = 1 if lps is None else lps * w.steps_per_cycle
    launch_t = fc_mean / launches_fc
    flops = spec["flops"] * pts * w.steps_per_cycle / launches_fc
    achieved = flops / launch_t / 1e12
    peak = alu["fp32_tflops"]
    hbm_bytes = spec.get("bytes", 2 * w.V * 4) * pts * w.steps_per_cycle / launches_fc
    hbm_achieved = hbm_bytes / launch_t / 1e9
    # dram__bytes_read.sum + dram__bytes_write.sum of one launch of the current
    # forecast kernel, from an ncu capture of this workload; None until
    # captured, and reset whenever the kernel changes
    traffic = spec["traffic"]
    g.close()

    if dist.rank == 0:
        line = {
            "metric": METRIC[args.workload],
            "value": value, "unit": "cycles/s", "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "nf": w.nf, "nc": w.nc, "ne": w.ne, "ny": w.ny,
                       "steps_per_cycle": w.steps_per_cycle, "precision": "mixed",
                       "gain_form": "ensemble-space", "replicas": dist.world,
                       "final_fine_iteration": args.regularise if args.regularise is not None else "off",
                       "l2": "flushed between timed cycles (256 MB write)",
                       **({"forecast_layout": _layout(M, fc_choice)} if args.workload == "ns2d" else {})},
            "member_steps_per_s": value * w.ne * w.steps_per_cycle,
            "forecast_ms_per_cycle": fc_mean * 1e3,
            "analysis_ms_per_cycle": (t_total / args.steps - fc_mean) * 1e3,
            "hbm_gbs_algorithmic": (2 * 4 * w.V * pts) * args.steps / t_total / 1e9,
            "fp64_plain": fp64_plain,
            "rmse_final": float(rmse_mixed[-1]),
            "regularisation": regularisation,
            "recentre_ablation": feedback,
            "filter_ablation": filt,
            "roofline": {"bound": "alu", "kernel": spec["kernel"],
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": "FP32 FMA throughput measured by mgk_fma_probe in this run (" +
                                        alu["how"] + ")",
                         "flops_per_point_step": spec["flops"],
                         "hbm_view": {"achieved_gbs": hbm_achieved, "peak_gbs": peaks.get("hbm_gbs"),
                                      "frac": hbm_achieved / float(peaks.get("hbm_gbs", 6800.0)),
                                      "bytes_per_point_step": hbm_bytes / (pts * w.steps_per_cycle / launches_fc),
                                      "peak_source": peak_src}},
            "alu_peaks": alu,
            "clocks": clk,
            "gpu_launches": int(launches),
            "wall_s_timed": wall,
        }
        if e2e:
            line["e2e"] = e2e
        if not args.no_cpu_baseline:
            import oracle as O
            O.build()
            line["cpu_baseline"] = cpu_baseline(w, inp)
        print(json.dumps(line), flush=True)


METRIC = {
    "burgers_large": "MGEnKF analysis cycles/s (1-D Burgers 16384/4096, Ne=128, 512 obs)",
    "ns2d": "MGEnKF analysis cycles/s (2-D NS 512^2/128^2, Ne=64, 2048 obs)",
    "ns2d_cnn": "MGEnKF analysis cycles/s with learned prolongation (2-D NS 1024^2/256^2, Ne=64)",
    "batched": "MGEnKF problem-cycles/s (96 independent 2-D NS problems, coarse 64^2..192^2, fine x4, "
               "Ne 16..128, 256..2048 obs, one graph launch per cycle)",
    "dual": "Dual MGEnKF analysis cycles/s with inlet-parameter estimation (Burgers inlet, 800 fine nodes, "
            "ratio 4, Ne=100, 80 sensors)",
}


# --------------------------------------------------------------------------
# Dual EnKF parameter estimation on the Burgers inlet model (Sec. 4 setting)
# --------------------------------------------------------------------------
DUAL = dict(nf=800, length=10.0, dt=2e-4, nu=1 / 200, ne=100, sigma=0.05, q=1e-6, nsteps=30, spin=50000,
            theta_true=(0.2, 0.0), theta_fine0=(0.0, 0.3))


def dual_inputs(seed):
    rng = np.random.default_rng(seed)
    ne = DUAL["ne"]
    theta0 = np.stack([rng.normal(0.0, 0.05, ne), rng.normal(0.3, 0.05, ne)], axis=1)
    return rng, theta0, np.arange(1, 81)


def dual_truth_obs(M, ncyc, rng, obs):
    """Observations of the truth run (theta = (0.2, 0), the fine model) for
    ncyc cycles after the spin-up, each with N(0, sigma^2) noise: a one-member
    dual object's fine run, advanced freely."""
    d = DUAL
    tr = M.DualMGEnKF(d["nf"], 1, 2, obs, d["length"], d["dt"], d["nu"], d["sigma"], 0.0, 1)
    tr.set_state(np.ones(d["nf"]), np.ones((2, d["nf"])), np.zeros((2, 2)), d["theta_true"], 0.0)
    tr.free_run(d["spin"])
    ys = np.empty((ncyc, obs.size))
    for k in range(ncyc):
        tr.free_run(d["nsteps"])
        ys[k] = tr.get_state()[0][obs] + d["sigma"] * rng.standard_normal(obs.size)
    tr.close()
    return ys


def run_gpu_dual(args, dist):
    import torch
    from paper_2012_10091_gb300 import mgenkf as M
    d = DUAL
    torch.cuda.set_device(dist.local)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    ncyc = args.warmup + args.steps
    nest = 500                                   # cycles of the parameter-estimation runs (3 t_c)
    rng, theta0, obs = dual_inputs(dist.rank)
    ys = dual_truth_obs(M, max(ncyc, nest), rng, obs)
    yd = torch.tensor(ys, dtype=torch.float64, device="cuda")

    def fresh(r):
        g = M.DualMGEnKF(d["nf"], r, d["ne"], obs, d["length"], d["dt"], d["nu"], d["sigma"], d["q"], 7,
                         stream=sp)
        g.set_state(np.ones(d["nf"]), np.ones((d["ne"], d["nf"] // r)), theta0, d["theta_fine0"], 0.0)
        g.free_run(d["spin"])
        return g

    g = fresh(4)
    for k in range(args.warmup):
        g.cycle(d["nsteps"], yd[k])
    torch.cuda.synchronize()
    dev = torch.cuda.current_device()
    clocks = ClockSampler(dev)
    clocks.start()
    n0 = M.mgk_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    e0.record(stream)
    for j in range(args.steps):
        g.cycle(d["nsteps"], yd[args.warmup + j])
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = M.mgk_kernel_launches() - n0
    t = dist.max(e0.elapsed_time(e1) / 1e3)
    g.close()
    # end to end: host observations in, the analysed parameter mean out, every cycle
    ge = fresh(4)
    th = np.empty(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(args.steps):
        ge.cycle(d["nsteps"], ys[j])
        M.lib.mgenkf_dual_get_state(ge.h, None, None, None, th.ctypes.data)
    te = dist.max(time.perf_counter() - t0)
    ge.close()
    # parameter estimates over 3 t_c for the paper's coarsening ratios
    est = {}
    for r in (1, 2, 4, 8, 16):
        ga = fresh(r)
        hist = np.empty((nest, 2))
        for k in range(nest):
            ga.cycle(d["nsteps"], yd[k])
            if k >= nest - 100:
                M.lib.mgenkf_dual_get_state(ga.h, None, None, None, hist[k].ctypes.data)
        ga.close()
        est[str(r)] = hist[-100:].mean(axis=0).tolist()
    cpu = None
    if dist.rank == 0 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        mg = O.DualMGEnKF(d["nf"], 4, d["length"], d["dt"], d["nu"], np.ones(d["nf"]), np.ones((d["ne"], d["nf"] // 4)),
                          theta0, d["theta_fine0"], obs, d["sigma"], 7, d["q"])
        mg.free_run(3000)
        nc_cpu = 20
        t0 = time.perf_counter()
        for k in range(nc_cpu):
            mg.cycle_step(d["nsteps"], ys[k])
        tc = time.perf_counter() - t0
        cpu = {"value": nc_cpu / tc, "unit": "cycles/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{nc_cpu} cycles of the ratio-4 dual run after 3000 free-run steps, OpenMP over members"}
    if dist.rank == 0:
        line = {"metric": METRIC["dual"], "value": dist.sum(args.steps) / t, "unit": "cycles/s",
                "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "burgers_inlet_800_r4_ne100_dual", "nf": d["nf"], "ratio": 4,
                           "ne": d["ne"], "ny": int(obs.size), "steps_per_cycle": d["nsteps"],
                           "theta_q": d["q"], "spin_up_steps": d["spin"],
                           "l2": "not flushed: the working set (< 2 MB) lives in L2 by design"},
                "theta_true": list(d["theta_true"]),
                "theta_estimate_last_100_of_500_cycles": est,
                "roofline": None,
                "roofline_note": "latency-bound: 800-node grids, one CTA each; see DESIGN",
                "clocks": clk, "gpu_launches": int(launches),
                "e2e": {"value": args.steps / te, "unit": "cycles/s", "h2d_bytes_per_step": 8 * int(obs.size),
                        "d2h_bytes_per_step": 16},
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)



# --------------------------------------------------------------------------
# batched workload: 96 independent NS-2D problems, sharded over ranks
# --------------------------------------------------------------------------
def problem_work(w) -> int:
    """Forecast points per model step (members and fine run) of one problem."""
    return w.ne * w.nc ** 2 + w.nf ** 2


def shard_problems(ws, world: int, rank: int) -> list:
    """Indices of the problems rank `rank` owns: greedy balance of the
    forecast work (largest first onto the least-loaded rank)."""
    work = [problem_work(w) for w in ws]
    load = [0] * world
    owner = [0] * len(ws)
    for i in sorted(range(len(ws)), key=lambda i: (-work[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += work[i]
    return [i for i in range(len(ws)) if owner[i] == rank]


def batched_cpu_estimate(ws, step_fraction: int):
    """Oracle time of one cycle of all problems, estimated from one sampled
    problem per coarse size (1/step_fraction of its forecast steps plus a full
    analysis, prolongation and RMSE), scaled to each problem by its forecast
    work.  Returns (seconds per batch cycle, description of the sample)."""
    import oracle as O
    from paper_2012_10091_gb300 import workloads as W
    per_nc = {}
    for w in ws:
        if w.nc in per_nc:
            continue
        inp = W.make_inputs(w)
        mg = O.MGEnKF(w.model, w.nf, w.ratio, w.length, w.dt, inp["fine0"], inp["members0"], inp["obs_idx"],
                      inp["obs_var"], w.sigma, w.seed, nu=w.nu, gamma=w.gamma, prandtl=w.prandtl)
        per_nc[w.nc] = (oracle_cycle_sample(w, inp, mg, step_fraction), problem_work(w), w.ne)
    t = sum(per_nc[w.nc][0] * problem_work(w) / per_nc[w.nc][1] for w in ws)
    desc = (f"one problem per coarse size ({', '.join(f'{nc}^2 Ne={v[2]}' for nc, v in sorted(per_nc.items()))}): "
            f"{max(1, 10 // step_fraction)} of 10 RK3 steps (time scaled) plus a full FP64 analysis, "
            f"prolongation and RMSE; each of the {len(ws)} problems scaled by its forecast points")
    return t, desc


def run_reference_batched(args, dist):
    if dist.rank != 0:
        return
    import oracle as O
    O.build()
    from paper_2012_10091_gb300 import workloads as W
    ws = W.ns2d_batch(args.problems, seed=0)
    times, desc = [], ""
    for j in range(args.warmup + args.steps):
        t, desc = batched_cpu_estimate(ws, 10)
        if j >= args.warmup:
            times.append(t)
    per = float(np.mean(times))
    val = len(ws) / per
    line = {"metric": METRIC["batched"], "value": val, "unit": "problem-cycles/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"ns2d_batch{len(ws)}_seed0", "problems": len(ws), "steps_per_cycle": 10,
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": "problem-cycles/s", "kind": "oracle", "cores": cpu_threads(),
                             "sample": desc},
            "e2e": {"value": val, "unit": "problem-cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu_batched(args, dist):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_10091_gb300 import mgenkf as M
    from paper_2012_10091_gb300 import workloads as W

    dev = dist.local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    ws_all = W.ns2d_batch(args.problems, seed=0)
    mine = shard_problems(ws_all, dist.world, dist.rank)
    ws = [ws_all[i] for i in mine]
    ncyc = args.warmup + args.steps
    nsteps = 10

    # handles (inputs generated and uploaded one problem at a time)
    runs, layouts, truth0 = [], [], []
    for w in ws:
        inp = W.make_inputs(w)
        g = M.MGEnKF.from_workload(w, stream=sp)
        g.set_state(inp["fine0"], inp["members0"])
        runs.append(g)
        layouts.append((inp["obs_idx"], inp["obs_var"]))
        truth0.append(inp["truth0"])
        del inp
    torch.cuda.synchronize()

    # synthetic observations: FP32 truth runs (one forecast per fine size),
    # sampled at each problem's probes plus N(0, sigma^2) noise; resident in HBM
    ny_tot = sum(w.ny for w in ws)
    yos = torch.empty((ncyc, ny_tot), dtype=torch.float64, device="cuda")
    by_nf = {}
    for j, w in enumerate(ws):
        by_nf.setdefault(w.nf, []).append(j)
    truths = {nf: torch.tensor(np.stack([truth0[j] for j in js]), dtype=torch.float32, device="cuda")
              for nf, js in by_nf.items()}
    off = np.cumsum([0] + [w.ny for w in ws])
    gidx = {}
    for nf, js in by_nf.items():
        rows = []
        for q, j in enumerate(js):
            oi, ov = layouts[j]
            rows.append(torch.tensor(q * 4 * nf * nf + ov.astype(np.int64) * nf * nf + oi, device="cuda"))
        gidx[nf] = rows
    with torch.cuda.stream(stream):
        for k in range(ncyc):
            for nf, js in by_nf.items():
                w0 = ws[js[0]]
                M.mgk_forecast(M.MGENKF_NS2D, M.MGENKF_MIXED, truths[nf], len(js), nf, w0.length, w0.dt, w0.nu,
                               w0.gamma, w0.prandtl, nsteps=nsteps, stream=sp)
                flat = truths[nf].view(-1)
                for q, j in enumerate(js):
                    yos[k, off[j]:off[j + 1]] = flat[gidx[nf][q]].double()
            noise = np.concatenate([W.observation_noise(w, k) for w in ws])
            yos[k] += torch.tensor(noise, device="cuda")
    torch.cuda.synchronize()
    del truths

    b = M.Batch(runs, stream=sp)
    t_tune = time.perf_counter()
    if args.tiles and os.path.exists(args.tiles):
        b.load_tiles(args.tiles)
        tuned = "loaded"
    else:
        b.autotune(reps=3)
        tuned = "autotuned"
        if args.tiles:
            b.save_tiles(args.tiles)
    t_tune = time.perf_counter() - t_tune
    tiles = b.tiles()
    innov = torch.zeros((ncyc, len(ws)), dtype=torch.float64, device="cuda")
    launches0 = M.mgk_kernel_launches()
    b.cycle(nsteps, yos[0], innov[0])          # captures the graph
    launches_per_cycle = M.mgk_kernel_launches() - launches0
    for k in range(1, args.warmup):
        b.cycle(nsteps, yos[k], innov[k])
    assert b.sync() == 0

    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for j in range(args.steps):
        k = args.warmup + j
        b.cycle(nsteps, yos[k], innov[k])
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - wall0
    dist.barrier()
    clk = clocks.stop()
    st = b.sync()
    if st:
        raise RuntimeError(f"batched run: device status {st}")
    t_total = e0.elapsed_time(e1) / 1e3
    t_max = dist.max(t_total)
    pc_all = dist.sum(float(len(ws) * args.steps))
    value = pc_all / t_max
    innov_h = innov.cpu().numpy()

    # forecast alone (all problems, one cycle's steps), for the stencil roofline
    fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    b.forecast(nsteps)
    fa.record(stream)
    for _ in range(reps):
        b.forecast(nsteps)
    fb.record(stream)
    torch.cuda.synchronize()
    fc_s = fa.elapsed_time(fb) / 1e3 / reps
    spec = WORKLOADS["batched"]
    pts = sum(problem_work(w) for w in ws)
    sizes = sorted(set(w.nc for w in ws) | set(w.nf for w in ws))
    n_launch = nsteps * len(sizes)
    peaks, peak_src = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    alu = measure_alu_peaks(M, torch, stream)
    flops_fc = spec["flops"] * pts * nsteps
    bytes_fc = spec["bytes"] * pts * nsteps
    alu_achieved = flops_fc / fc_s / 1e12
    hbm_achieved = bytes_fc / fc_s / 1e9

    # e2e: observations from pinned host memory, innovation RMS read back each cycle
    e2e = None
    if not args.no_e2e:
        y_h = torch.empty((ncyc, ny_tot), dtype=torch.float64, pin_memory=True)
        y_h.copy_(yos.cpu())
        o_h = torch.empty((ncyc, len(ws)), dtype=torch.float64, pin_memory=True)
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in range(args.steps):
            k = args.warmup + j
            b.cycle(nsteps, y_h[k], o_h[k])
            stream.synchronize()                     # the cycle's innovation RMS is on the host
        te = dist.max(time.perf_counter() - t0)
        assert b.sync() == 0
        e2e = {"value": pc_all / te, "unit": "problem-cycles/s", "h2d_bytes_per_step": 8 * ny_tot,
               "d2h_bytes_per_step": 8 * len(ws)}

    # plain FP64 against mixed precision on one problem per coarse size, lockstep
    # with an FP64 truth run, RMSE of the fine run
    fp64 = None
    if args.fp64_cycles > 0 and dist.rank == 0:
        sample = {}
        for w in ws_all:
            sample.setdefault(w.nc, w)
        rows = []
        for nc, w in sorted(sample.items()):
            inp = W.make_inputs(w)
            g64 = M.MGEnKF.from_workload(w, precision="fp64", stream=sp)
            gm = M.MGEnKF.from_workload(w, precision="mixed", stream=sp)
            for g in (g64, gm):
                g.set_state(inp["fine0"], inp["members0"])
            tr = torch.tensor(inp["truth0"], dtype=torch.float64, device="cuda")
            idx = torch.tensor(inp["obs_var"].astype(np.int64) * w.nf ** 2 + inp["obs_idx"], device="cuda")
            r64 = torch.zeros((args.fp64_cycles, 4), dtype=torch.float64, device="cuda")
            rmx = torch.zeros_like(r64)
            ta, tb, tc = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            t64 = tmx = 0.0
            with torch.cuda.stream(stream):
                for k in range(args.fp64_cycles):
                    M.mgk_forecast(M.MGENKF_NS2D, M.MGENKF_FP64, tr, 1, w.nf, w.length, w.dt, w.nu, w.gamma,
                                   w.prandtl, nsteps=nsteps, stream=sp)
                    yo = tr[idx] + torch.tensor(W.observation_noise(w, k), device="cuda")
                    ta.record(stream)
                    M.mgenkf_cycle(g64.h, nsteps, yo, tr, r64[k])
                    tb.record(stream)
                    M.mgenkf_cycle(gm.h, nsteps, yo, tr, rmx[k])
                    tc.record(stream)
                    tc.synchronize()
                    t64 += ta.elapsed_time(tb)
                    tmx += tb.elapsed_time(tc)
            assert g64.sync() == 0 and gm.sync() == 0
            half = slice(args.fp64_cycles // 2, args.fp64_cycles)
            a, m_ = float(r64[half, 0].mean()), float(rmx[half, 0].mean())
            rows.append({"problem": w.name, "rmse_fp64": a, "rmse_mixed": m_, "rmse_rel_diff": abs(m_ - a) / a,
                         "fp64_ms_per_cycle": t64 / args.fp64_cycles, "mixed_ms_per_cycle": tmx / args.fp64_cycles})
            g64.close()
            gm.close()
        fp64 = {"cycles": args.fp64_cycles, "problems": rows,
                "max_rmse_rel_diff": max(r["rmse_rel_diff"] for r in rows)}

    b.close()
    for g in runs:
        g.close()

    if dist.rank == 0:
        line = {
            "metric": METRIC["batched"], "value": value, "unit": "problem-cycles/s", "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"ns2d_batch{len(ws_all)}_seed0", "problems": len(ws_all),
                       "problems_rank0": len(ws), "steps_per_cycle": nsteps, "precision": "mixed",
                       "gain_form": "ensemble-space", "segment_rows": {str(k): M.SEGMENT_ROWS[v] for k, v in
                                                                sorted(tiles.items())},
                       "narrow_bands": [k for k, v in sorted(tiles.items()) if M.NARROW_BANDS[v]],
                       "tile_table": tuned, "autotune_s": t_tune,
                       "l2": f"not flushed: working set {sum(4 * 4 * (3 * problem_work(w)) for w in ws) / 1e9:.2f} GB "
                             f"(states + stage buffers) > L2 (129 MB)"},
            "batch_cycles_per_s": args.steps / t_total,
            "member_steps_per_s": value / len(ws_all) * sum(w.ne for w in ws_all) * nsteps,
            "forecast_ms_per_cycle": fc_s * 1e3,
            "analysis_ms_per_cycle": (t_total / args.steps - fc_s) * 1e3,
            "kernels_per_cycle": int(launches_per_cycle),
            "innovation_rms_mean_last": float(innov_h[-1].mean()),
            # the forecast's launches (one per model step and grid size, the
            # sizes on concurrent streams) timed as one unit by CUDA events on
            # the batch stream: algorithmic flops (FP32 view) and bytes (HBM
            # view) of all of them over that time; bound = the larger fraction
            "roofline": {"bound": "alu", "kernel": spec["kernel"], "achieved": alu_achieved,
                         "peak": alu["fp32_tflops"], "unit": "TFLOP/s", "frac": alu_achieved / alu["fp32_tflops"],
                         "traffic": (spec["traffic_per_point_step"] * pts * nsteps
                                     if spec.get("traffic_per_point_step") else None),
                         "scope": f"all march launches of one forecast ({n_launch} launches: {nsteps} steps x "
                                  f"{len(sizes)} grid sizes), {pts * nsteps / 1e9:.3f} G point-steps, "
                                  f"{spec['flops']} flops and {spec['bytes']} B per point-step",
                         "peak_source": "FP32 FMA throughput measured by mgk_fma_probe in this run (" +
                                        alu["how"] + ")",
                         "hbm_view": {"achieved_gbs": hbm_achieved, "peak_gbs": hbm_peak,
                                      "frac": hbm_achieved / hbm_peak, "peak_source": f"hbm_gbs ({peak_src})"}},
            "alu_peaks": alu,
            "fp64_plain": fp64,
            "clocks": clk,
            "gpu_launches": int(launches_per_cycle * args.steps),
            "wall_s_timed": wall,
        }
        if e2e:
            line["e2e"] = e2e
        if not args.no_cpu_baseline:
            import oracle as O
            O.build()
            t, desc = batched_cpu_estimate(ws_all, 10)
            line["cpu_baseline"] = {"value": len(ws_all) / t, "unit": "problem-cycles/s", "cores": cpu_threads(),
                                    "kind": "oracle", "sample": desc}
        print(json.dumps(line), flush=True)


def run_gpu_cnn(args, dist, w, inp):
    """Learned-correction configuration: train on pairs from lockstep MGEnKF /
    full-resolution EnKF runs (untimed), then time cycles with the network
    attached to prolong_correct, and cycles with plain prolongation."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_10091_gb300 import mgenkf as M
    from paper_2012_10091_gb300 import surrogate as S
    from paper_2012_10091_gb300 import workloads as W

    dev = dist.local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    per_seed = 200
    sets, seed = [], 100 + dist.rank * 1000
    while sum(s_["dC"].shape[0] for s_ in sets) < args.cnn_pairs:
        n = min(per_seed, args.cnn_pairs - sum(s_["dC"].shape[0] for s_ in sets))
        ws = W.ns2d_shear(nf=w.nf, ratio=w.ratio, ne=w.ne, n_probes=w.n_probes, precision="mixed", seed=seed)
        sets.append(S.generate_pairs(ws, n))
        seed += 1
    t_gen = time.perf_counter() - t0
    train = S.concat_pairs(*sets[:-1]) if len(sets) > 1 else sets[0]
    val = sets[-1] if len(sets) > 1 else None
    t1 = time.perf_counter()
    cnn, stats, hist = S.fit(train, epochs=args.cnn_epochs, batch=8, lr=3e-4, val_pairs=val)
    t_fit = time.perf_counter() - t1
    del sets, train, val
    torch.cuda.empty_cache()

    ncyc = args.warmup + args.steps
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    with torch.cuda.stream(stream):
        truths, yos = truth_and_obs(M, w, inp, ncyc, torch, "fp64")
    torch.cuda.synchronize()
    res = {}
    for mode in ("cnn", "plain"):
        g = M.MGEnKF.from_workload(w, stream=sp)
        g.set_state(inp["fine0"], inp["members0"])
        if mode == "cnn":
            fc_choice = _forecast_choice(g, args)
            g.set_prolong_cnn(cnn)
        else:
            g.set_forecast_choice(*fc_choice)
        rm = torch.zeros((ncyc, w.V), dtype=torch.float64, device="cuda")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for k in range(args.warmup):
                M.mgenkf_cycle(g.h, w.steps_per_cycle, yos[k], truths[k], rm[k])
        torch.cuda.synchronize()
        dist.barrier()
        clocks = ClockSampler(dev)
        clocks.start()
        launches0 = M.mgk_kernel_launches()
        with torch.cuda.stream(stream):
            for j in range(args.steps):
                k = args.warmup + j
                e0, e1, e2 = ev[j]
                e0.record(stream)
                M.mgenkf_forecast(g.h, w.steps_per_cycle)
                M.mgenkf_analyse(g.h, yos[k])
                e1.record(stream)
                M.mgenkf_prolong_correct(g.h)
                M.mgenkf_rmse(g.h, truths[k], rm[k])
                e2.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        assert g.sync() == 0
        tot = dist.max(sum(a.elapsed_time(c) for a, _, c in ev) / 1e3)
        res[mode] = dict(cps=dist.sum(float(args.steps)) / tot, ms=tot / args.steps * 1e3,
                         prolong_ms=float(np.mean([b.elapsed_time(c) for _, b, c in ev])),
                         rmse=rm[ncyc // 2:].mean(0).cpu().numpy().tolist(), clocks=clk,
                         launches=int(M.mgk_kernel_launches() - launches0))
        g.close()
    cnn.close()
    if dist.rank == 0:
        cnn_flops = CNN_FLOPS_PER_PIXEL * w.nc ** 2
        line = {
            "metric": METRIC[args.workload], "value": res["cnn"]["cps"], "unit": "cycles/s",
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["cnn"]["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name + "_cnn", "nf": w.nf, "nc": w.nc, "ne": w.ne, "ny": w.ny,
                       "steps_per_cycle": w.steps_per_cycle, "precision": "mixed",
                       "prolongation": "Pi_F + learned residual (BF16 CNN, 30080 parameters)",
                       "training_pairs": args.cnn_pairs, "epochs": args.cnn_epochs,
                       "forecast_layout": _layout(M, fc_choice),
                       "l2": "inputs larger than L2 (fine state 16 MB, members 67 MB per cycle step)"},
            "plain_prolongation": {"cycles_per_s": res["plain"]["cps"],
                                   "prolong_ms": res["plain"]["prolong_ms"],
                                   "rmse_last_half": res["plain"]["rmse"]},
            "cnn": {"prolong_ms": res["cnn"]["prolong_ms"], "rmse_last_half": res["cnn"]["rmse"],
                    "val_loss": min(hist["val"]) if hist["val"] else None,
                    "val_loss_plain": hist["val_plain"], "gen_s": t_gen, "fit_s": t_fit,
                    "inference_gflop": cnn_flops / 1e9,
                    "inference_tflops": cnn_flops / (res["cnn"]["prolong_ms"] - res["plain"]["prolong_ms"]) / 1e9
                    if res["cnn"]["prolong_ms"] > res["plain"]["prolong_ms"] else None},
            "clocks": res["cnn"]["clocks"], "gpu_launches": res["cnn"]["launches"],
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    dist = Dist()
    from paper_2012_10091_gb300 import workloads as W
    if args.workload == "batched":
        try:
            if args.impl == "reference":
                run_reference_batched(args, dist)
            else:
                run_gpu_batched(args, dist)
        finally:
            dist.close()
        return
    if args.workload == "dual":
        try:
            run_gpu_dual(args, dist)
        finally:
            dist.close()
        return
    if args.workload == "ns2d_cnn":
        w = W.ns2d_shear(nf=1024, ratio=4, ne=64, n_probes=1024, seed=dist.rank)
    elif args.workload == "ns2d":
        w = W.ns2d_shear(seed=dist.rank)
    else:
        w = W.burgers_large(seed=dist.rank)
    inp = W.make_inputs(w)
    try:
        if args.impl == "reference":
            run_reference(args, dist, w, inp)
        elif args.workload == "ns2d_cnn":
            run_gpu_cnn(args, dist, w, inp)
        else:
            run_gpu(args, dist, w, inp)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
