"""Benchmark: time to 1e-10 relative residual of nonstandard-coarsening multigrid.

Workload (one step): 2D Poisson, fourth-order 9-point Laplacian on 4097 x 4097
nodes (N = 4096), FP64, right-hand side = 16 seeded sin(k pi x) sin(l pi y)
modes (k, l uniform in 1..64, amplitudes N(0,1)), red-black coarsening down to a
3 x 3 grid, Galerkin coarse operators built from the second-order operator
(G^(2)), V(2,1) cycles with red-black smoothing, solved from u = 0 until
||f - L u|| / ||f|| < 1e-10. The non-Galerkin and standard-coarsening runs of
the same workload are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0). Multi-GPU runs are independent replicas.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-10 rel. residual and HBM GB/s, mixed vs FP64; p50/p99 served latency"
N = 4096
ORDER = 4
RTOL = 1e-10
NU1, NU2 = 2, 1
SEED = 0
WORKLOAD = ("2D Poisson -Lap u = f, 4th-order 9-point Laplacian, 4097x4097 nodes (N=4096), FP64; "
            "f = 16 seeded sin*sin modes (freq 1-64, N(0,1) amplitudes); red-black coarsening to 3x3, "
            "Galerkin G^(2) coarse operators, V(2,1) red-black smoothing, omega=1, solve from u=0 to 1e-10")

# DRAM bytes (read + write) per launch of the dominant kernel, k_half_sweep_nt<double,
# exact, 9> on level 0, from one ncu capture of `bench.py --profile-case` (the summary
# under profiles/ names the kernel and workload); None whenever that kernel changes.
DOMINANT_KERNEL_TRAFFIC_BYTES = 373.25e6

# The batched and served problems stop coarsening at a 16-cell axis grid and solve its
# 225 unknowns exactly with the dense factor (fewer near-empty small levels); the
# headline workload coarsens to one unknown.
N_MIN_SMALL = 16

# FP64 peak of GB300: 1.25 TFLOP/s nominal (an FMA counts two flops). MEASURED_PEAKS.json
# carries no FP64 figure; the measured DFMA issue rate (600 G/s, 1.20 TFLOP/s) is quoted
# beside it. Flops per updated node of a half-sweep: 2 s for the stencil application of
# s terms plus 3 (f - L u, the multiply by omega / a_pp, the add to u): 21 for s = 9.
FP64_PEAK_TFLOPS = 1.25
FP64_DFMA_MEASURED_TFLOPS = 1.1998  # python bench.py --fp-pipe-probe (DFMA line x 2 flops)

# Issue-rate probe behind FP64_DFMA_MEASURED_TFLOPS: per thread, 8 independent chains of
# one instruction kind (no memory traffic); one warm-up launch, then the mean of 5
# launches timed with CUDA events.
FP_PIPE_PROBE_CU = r"""// Floating-point pipe throughput probe for the ALU roofline of the FP64 kernels:
// independent FMA / add / multiply chains per thread, no memory traffic.
#include <cstdio>
#include <cuda_runtime.h>
template <int OP, typename T>
__global__ void k(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (OP == 0) x[c] = fma(x[c], a, b);
      else if (OP == 1) x[c] = x[c] + b;
      else x[c] = x[c] * a;
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <int OP, typename T>
void run(const char* name, T a, T b) {
  int blocks = 152 * 8, threads = 256, iters = 2048;
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  k<OP, T><<<blocks, threads>>>(out, iters, a, b);
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  for (int r = 0; r < 5; ++r) k<OP, T><<<blocks, threads>>>(out, iters, a, b);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  double ops = 5.0 * blocks * threads * (double)iters * 8;
  printf("%s: %.1f Gop/s (%.3f ms per launch) err=%s\n", name, ops / (ms * 1e-3) / 1e9, ms / 5,
         cudaGetErrorString(cudaGetLastError()));
  cudaFree(out);
}
int main() {
  int clk; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  printf("SMs %d, clock %d kHz\n", sms, clk);
  run<0, double>("DFMA", 0.999999, 1e-7);
  run<1, double>("DADD", 0.999999, 1e-7);
  run<2, double>("DMUL", 0.999999, 1e-7);
  run<0, float>("FFMA", 0.999999f, 1e-7f);
  run<1, float>("FADD", 0.999999f, 1e-7f);
  return 0;
}
"""


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    """Largest value over all ranks (the slowest replica sets the step time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_cores():
    """Cores this process may run on, and the machine's core count."""
    try:
        usable = len(os.sched_getaffinity(0))
    except Exception:
        usable = os.cpu_count()
    return usable, os.cpu_count()


def build_oracle(n: int = N):
    """The FP64 oracle of the bench workload on an (n+1)^2 grid, its right-hand side, and
    the seconds the build took."""
    import synth
    from oracle.mg import GALERKIN, REDBLACK, Options, Oracle
    t0 = time.perf_counter()
    o = Oracle(n, ORDER, REDBLACK, GALERKIN, Options(nu1=NU1, nu2=NU2))
    setup_s = time.perf_counter() - t0
    return o, o.to_vec(synth.rhs_sine_modes(n, SEED)), setup_s


def oracle_cycle_times(o, f, cycles: int, residuals: int = 0):
    """Time `cycles` consecutive V(2,1) cycles of the oracle from u = 0 (each from the
    previous iterate); the relative residual after each of the first `residuals` cycles
    is evaluated outside the timed region. Returns (seconds per cycle, residual history)."""
    import numpy as np
    u = np.zeros_like(f)
    hist = [o.rel_residual(u, f)]
    times = []
    for k in range(cycles):
        t0 = time.perf_counter()
        u = o.cycle(u, f)
        times.append(time.perf_counter() - t0)
        if k < residuals:
            hist.append(o.rel_residual(u, f))
    # the cycle count to the tolerance, if the timed cycles did not reach it (not timed)
    while residuals and hist[-1] >= RTOL and len(hist) <= 30:
        u = o.cycle(u, f)
        hist.append(o.rel_residual(u, f))
    return times, hist


def _all_cores_worker(n):
    o, f, _ = build_oracle(n)
    times, _ = oracle_cycle_times(o, f, 1)
    return times[0]


def oracle_all_cores(n: int = 1024):
    """Every usable core runs its own oracle (one V(2,1) cycle on an (n+1)^2 grid of the
    workload, processes started with spawn): aggregate grid-point-cycles/s against one
    process alone. The oracle itself is single-threaded numpy/scipy."""
    import multiprocessing as mp
    usable, _ = host_cores()
    one = _all_cores_worker(n)
    ctx = mp.get_context("spawn")
    with ctx.Pool(usable) as pool:
        t0 = time.perf_counter()
        per = pool.map(_all_cores_worker, [n] * usable)
        wall = time.perf_counter() - t0
    pts = (n + 1) ** 2
    return {"processes": usable, "grid": f"{n + 1}^2", "cycle_s_one_process": one,
            "cycle_s_median_all_cores": statistics.median(per),
            "grid_point_cycles_per_s_one_process": pts / one,
            "grid_point_cycles_per_s_all_cores": usable * pts / statistics.median(per),
            "wall_s_including_setup": wall}


def run_reference(args, ws, rank):
    """The FP64 oracle on the host cores, on the bench workload itself (4097^2): built once
    (not timed), then every step is one oracle V(2,1) cycle continuing from the previous
    iterate. value = median cycle time x the cycles the oracle needs to reach 1e-10 (its
    own residual history, evaluated outside the timed cycles)."""
    if rank != 0:
        return
    o, f, setup_s = build_oracle(args.ref_n)
    times, hist = oracle_cycle_times(o, f, args.warmup + args.steps, residuals=min(12, args.warmup + args.steps))
    timed = times[args.warmup:]
    cyc_ms = statistics.median(timed) * 1e3
    below = [k for k, r in enumerate(hist) if r < RTOL]
    cycles = below[0] if below else None
    value = cyc_ms * cycles if cycles else None
    usable, total = host_cores()
    allc = None if args.no_all_cores else oracle_all_cores()
    sample = (f"one V(2,1) cycle of the oracle per step on the {args.ref_n + 1}^2 workload itself "
              f"(build {setup_s:.1f} s, not timed); value = median cycle time x {cycles} cycles to 1e-10 "
              f"(the oracle's own residual history)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": cyc_ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": "replicas", "step": "one oracle V(2,1) cycle",
                   "cycles_to_tol": cycles, "history": hist, "cycle_ms_all": [t * 1e3 for t in timed],
                   "setup_s": setup_s},
        "cpu_baseline": {"value": value, "unit": "ms", "cores": 1, "host_cores": total, "usable_cores": usable,
                         "kind": "oracle", "sample": sample, "all_cores": allc},
        "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    import paper_2008_03885_gb300 as mg
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    F = synth.rhs_sine_modes(N, SEED)
    f_host = torch.from_numpy(F).pin_memory()
    u_host = torch.zeros_like(f_host).pin_memory()
    f = f_host.to(dev)
    u = torch.zeros_like(f)
    bytes_grid = f.numel() * 8

    def solve(h, uu, ff):
        uu.zero_()
        k, hist = mg.mg_solve(h, uu, ff, rtol=RTOL, max_cycles=60)
        return k, hist

    h = mg.mg_setup(N, ORDER, "redblack", "galerkin", nu1=NU1, nu2=NU2)
    for _ in range(args.warmup):
        cycles, hist = solve(h, u, f)
    torch.cuda.synchronize()

    # ---- timed region: K solves, device time via events on the launching stream
    mg.mg_reset_counters(h)
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            cycles, hist = solve(h, u, f)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ws, ms)
    launches, ncyc = mg.mg_get_counters(h)
    clocks = clk.summary()

    # ---- per-kernel CUDA events: the same K solves again with event brackets around
    # every finest-level launch (events need eager launches, so this pass does not use
    # the cycle's CUDA graph; kernel durations are the same)
    mg.mg_set_timing(h, True)
    for _ in range(args.steps):
        solve(h, u, f)
    torch.cuda.synchronize()
    kt = {k: mg.mg_get_timing(h, k) for k in range(5)}
    mg.mg_set_timing(h, False)

    # ---- end to end through the C ABI with host buffers: mg_solve_host copies f and the
    # initial guess u from pinned host memory, solves, and copies u back, every step
    # (one zero-initialised pinned u per step, so no host work sits between the calls)
    u_steps = [torch.zeros_like(u_host).pin_memory() for _ in range(args.steps)]
    mg.mg_solve_host(h, torch.zeros_like(u_host).pin_memory(), f_host, rtol=RTOL, max_cycles=60,
                     stream=stream)  # first call allocates the handle's device copies
    barrier(ws)
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for k in range(args.steps):
        mg.mg_solve_host(h, u_steps[k], f_host, rtol=RTOL, max_cycles=60, stream=stream)
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(ws, e2.elapsed_time(e3) / args.steps)
    assert torch.equal(u_steps[-1], u.cpu()), "host-buffer solve differs from the device solve"
    final_rr = hist[-1]
    # the same host <-> device copies alone (pinned memory, the call's stream), to split
    # the end-to-end time into copies and solve
    dev_f, dev_u = torch.empty_like(f), torch.empty_like(u)
    cp = []
    for k in range(args.steps):
        a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a0.record(stream)
        dev_f.copy_(f_host, non_blocking=True)
        dev_u.copy_(u_steps[k], non_blocking=True)
        a1.record(stream)
        u_steps[k].copy_(dev_u, non_blocking=True)
        a2.record(stream)
        torch.cuda.synchronize()
        cp.append((a0.elapsed_time(a1), a1.elapsed_time(a2)))
    h2d_ms = statistics.median(c[0] for c in cp)
    d2h_ms = statistics.median(c[1] for c in cp)
    del dev_f, dev_u

    # ---- variants of the same workload (one timed solve each after one warm-up)
    variants = {}
    f_periodic = None  # zero-mean N(0,1) on the nodes 0 <= i, j < N (periodic variants)
    if not args.quick:
        for name, co, op, omega, extra in (
                ("redblack_nongalerkin", "redblack", "nongalerkin", 1.0, {}),
                ("standard_galerkin_omega1.1", "standard", "galerkin", 1.1, {}),
                ("fp64_fma_contract", "redblack", "galerkin", 1.0, {"fma_contract": 1}),
                ("fp64_dense_coarsest_nmin16", "redblack", "galerkin", 1.0, {"n_min": 16}),
                ("mixed_dense_coarsest_nmin16", "redblack", "galerkin", 1.0,
                 {"precision": mg.MG_PREC_MIXED_FP32, "inner_cycles": 1, "fma_contract": 1, "n_min": 16}),
                ("mixed_fp32_inner", "redblack", "galerkin", 1.0,
                 {"precision": mg.MG_PREC_MIXED_FP32, "inner_cycles": 1, "fma_contract": 1}),
                ("mixed_fp32_inner_nongalerkin_coarse", "redblack", "nongalerkin", 1.0,
                 {"precision": mg.MG_PREC_MIXED_FP32, "inner_cycles": 1, "fma_contract": 1}),
                ("standard_cubic_nongalerkin4_omega1.1", "standard", "nongalerkin_high", 1.1, {"transfer_order": 4}),
                ("periodic_redblack_galerkin", "redblack", "galerkin", 1.0, {"boundary": "periodic"}),
                ("periodic_mixed_fp32_inner", "redblack", "galerkin", 1.0,
                 {"boundary": "periodic", "precision": mg.MG_PREC_MIXED_FP32, "inner_cycles": 1,
                  "fma_contract": 1})):
            fv = f
            if extra.get("boundary") == "periodic":
                if f_periodic is None:
                    import synth
                    f_periodic = torch.tensor(synth.rhs_periodic_normal(N, seed=3), dtype=torch.float64,
                                              device=f.device)
                fv = f_periodic
            hv = mg.mg_setup(N, ORDER, co, op, nu1=NU1, nu2=NU2, omega=omega, **extra)
            solve(hv, u, fv)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            var_ms = []
            for _ in range(3):  # best of three timed solves (one solve is ~20-150 ms)
                a.record(stream)
                kv, hv_hist = solve(hv, u, fv)
                b.record(stream)
                torch.cuda.synchronize()
                var_ms.append(a.elapsed_time(b))
            mg.mg_set_timing(hv, True)  # kernel breakdown from a second, eagerly launched solve
            solve(hv, u, fv)
            torch.cuda.synchronize()
            vt = {nm: mg.mg_get_timing(hv, k) for k, nm in
                  enumerate(("smooth", "residual", "restrict", "prolong", "norm"))}
            variants[name] = {"ms": min(var_ms), "ms_all": var_ms, "cycles": kv, "final_rel_res": hv_hist[-1],
                              "cr_last": hv_hist[-1] / hv_hist[-2] if kv > 1 else None,
                              "boundary": extra.get("boundary", "dirichlet"),
                              "transfer_order": extra.get("transfer_order", 2),
                              "finest_kernel_ms": {k: v[0] for k, v in vt.items()},
                              "finest_kernel_launches": {k: v[1] for k, v in vt.items()}}
            hv.close()
    large = run_mixed_large(args) if not args.quick and not args.no_extras else None
    batched = run_batched(args) if not args.quick and not args.no_extras else None
    served = run_serving(args) if not args.quick and not args.no_extras else None

    # ---- roofline of the dominant kernel (finest-level red-black half-sweep, FP64)
    sm_ms, sm_n = kt[mg.MG_KERNEL_SMOOTH]
    per_launch_ms = sm_ms / max(sm_n, 1)
    pts = (N - 1) ** 2
    flops_per_launch = pts / 2 * (2 * 9 + 3)  # updated nodes x (2 s + 3), s = 9 terms
    bytes_per_launch = 12 * (N + 1) ** 2  # half of a sweep's 24 B per node (read u, f; write u)
    achieved_tflops = flops_per_launch / (per_launch_ms * 1e-3) / 1e12
    hbm_peak, peak_kind = load_peaks()
    achieved_gbs = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9
    total_kernel_ms = sum(v[0] for v in kt.values())
    out = {
        "metric": METRIC, "value": ms_max, "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "order": ORDER, "coarsening": "redblack",
                   "coarse_op": "galerkin (G^(2))", "cycle": f"V({NU1},{NU2})", "omega": 1.0, "rtol": RTOL,
                   "cycles_to_tol": cycles, "final_rel_res": final_rr, "fma_contract": 0,
                   "l2": "inputs larger than L2: f alone is 134 MB and the hierarchy ~1.1 GB per solve",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved_tflops / FP64_PEAK_TFLOPS,
                     "traffic": DOMINANT_KERNEL_TRAFFIC_BYTES, "algorithmic_bytes": bytes_per_launch,
                     "traffic_over_algorithmic": (DOMINANT_KERNEL_TRAFFIC_BYTES / bytes_per_launch
                                                  if DOMINANT_KERNEL_TRAFFIC_BYTES else None),
                     "algorithmic_flops": flops_per_launch,
                     "kernel": "k_half_sweep_nt<double, exact, 9> on level 0",
                     "per_launch_ms": per_launch_ms, "launches": sm_n,
                     "peak_kind": "FP64 1.25 TFLOP/s nominal (FMA = 2 flops); no FP64 figure in "
                                  "MEASURED_PEAKS.json",
                     "frac_of_measured_dfma_rate": achieved_tflops / FP64_DFMA_MEASURED_TFLOPS,
                     "note": "exact evaluation order (no FMA; each row's groups of equal coefficient summed "
                             "then multiplied): 14 DADD/DMUL per updated node for the method's 21 flops, issued "
                             "at most 0.506 T/s (measured), so this kernel cannot exceed 0.61 of the nominal "
                             "FP64 peak",
                     "fp64_ops_per_updated_node": 14,
                     "hbm_gbs_algorithmic": achieved_gbs, "hbm_frac_algorithmic": achieved_gbs / hbm_peak,
                     "hbm_peak_gbs": hbm_peak, "hbm_peak_kind": peak_kind,
                     "share_of_finest_level_kernel_time": sm_ms / total_kernel_ms if total_kernel_ms else None},
        "roofline_fp32_smoothing": fp32_smoothing_roofline(variants.get("mixed_fp32_inner"), hbm_peak, peak_kind),
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 2 * bytes_grid, "d2h_bytes_per_step": bytes_grid,
                "breakdown_ms": {"h2d_copies": h2d_ms, "d2h_copy": d2h_ms, "device_solve": ms_max,
                                 "rest": e2e_ms - h2d_ms - d2h_ms - ms_max},
                "copy_gbs": {"h2d": 2 * bytes_grid / (h2d_ms * 1e-3) / 1e9,
                             "d2h": bytes_grid / (d2h_ms * 1e-3) / 1e9}},
        "throughput": solve_throughput(ms_max, cycles, variants.get("mixed_fp32_inner")),
        "gpu_launches": launches,
        "clocks": clocks,
        "variants": variants,
        "mixed_vs_fp64_8193": large,
        "batched": batched,
        "serving": served,
        "kernel_ms_per_step": {name: kt[k][0] / args.steps for k, name in
                               enumerate(("smooth", "residual", "restrict", "prolong", "norm"))},
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        del u, f
        torch.cuda.empty_cache()
        o, fo, setup_s = build_oracle(N)
        times, _ = oracle_cycle_times(o, fo, 1)
        del o, fo
        usable, total = host_cores()
        out["cpu_baseline"] = {"value": times[0] * cycles * 1e3, "unit": "ms", "cores": 1, "host_cores": total,
                               "usable_cores": usable, "kind": "oracle",
                               "sample": f"one V(2,1) cycle of the oracle on the 4097^2 workload itself "
                                         f"({times[0]:.2f} s; build {setup_s:.1f} s, not timed) x {cycles} "
                                         f"cycles to 1e-10 (the oracle's iterates are bitwise the GPU's, so "
                                         f"it needs the same count)"}
    if rank == 0:
        print(json.dumps(out))


def fp32_smoothing_roofline(mixed, hbm_peak, peak_kind):
    """HBM roofline of the mixed path's level-0 FP32 red-black smoothing, on the method's
    algorithmic bytes: 12 B per node per full sweep (read u and f, write u once), i.e.
    6 B per node per half-sweep; V(2,1) makes 2 (nu1 + nu2) = 6 half-sweeps per
    refinement step on level 0. With the TMA tile kernels (4097^2) they run as two
    launches per step: the presmooth (nu1 sweeps from zero) and one post-smoothing
    sweep. Without them (per-half-sweep launches) the first red half-sweep runs inside
    the FP64 refinement residual (timed with the norm class), so the smoothing launches
    carry 5 of the 6."""
    if not mixed:
        return None
    sm_ms, sm_n = mixed["finest_kernel_ms"]["smooth"], mixed["finest_kernel_launches"]["smooth"]
    steps = mixed["cycles"]
    tiles = sm_n == 2 * steps
    half_sweeps = 2 * (NU1 + NU2) - (0 if tiles else 1)
    alg = steps * half_sweeps * 6 * (N + 1) ** 2
    gbs = alg / (sm_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
            "peak_kind": peak_kind, "algorithmic_bytes_per_solve": alg, "launches_per_solve": sm_n,
            "half_sweeps_per_step": half_sweeps, "tile_kernels": tiles, "ms_per_solve": sm_ms,
            "kernel": "level-0 FP32 smoothing of the mixed path (4097^2, order 4)"}


def run_mixed_large(args):
    """8193^2 (N = 8192), orders 2 and 4, N(0,1) right-hand side: time to 1e-10 of the
    FP64 path (exact evaluation order, bitwise equal to the oracle's iterates) and of
    the mixed path (FP32 inner cycles, FP64 refinement); each solution's relative error
    against the FP64 oracle's exact discrete solution (Fourier diagonalisation with the
    operator's symbol, oracle/spectral.py, computed on the host outside the timing) and
    the mixed solution's difference from the FP64 one."""
    import torch
    import paper_2008_03885_gb300 as mg
    import synth
    from oracle import spectral
    n = args.large_n
    F = synth.rhs_normal(n, SEED + 3)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    out = {"n": n, "rhs": "N(0,1) i.i.d.", "rtol": RTOL,
           "error_reference": "oracle exact discrete solution (oracle/spectral.py: DST-I with the symbol)"}
    for order in (2, 4):
        res = {}
        sols = {}
        t0 = time.perf_counter()
        U = torch.tensor(spectral.solve(F, order, workers=-1), dtype=torch.float64, device="cuda")
        oracle_s = time.perf_counter() - t0
        for name, extra in (("fp64", {}), ("mixed", {"precision": mg.MG_PREC_MIXED_FP32, "fma_contract": 1})):
            h = mg.mg_setup(n, order, "redblack", "galerkin", nu1=NU1 if order == 4 else 1, nu2=1, **extra)
            u = torch.zeros_like(f)
            mg.mg_solve(h, u, f, rtol=RTOL, max_cycles=60)  # warm-up (graph capture)
            torch.cuda.synchronize()
            u.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            k, hist = mg.mg_solve(h, u, f, rtol=RTOL, max_cycles=60)
            b.record(stream)
            torch.cuda.synchronize()
            h.close()
            res[name] = {"ms": a.elapsed_time(b), "cycles": k, "final_rel_res": hist[-1]}
            sols[name] = u
        err = float(torch.linalg.norm(sols["mixed"] - sols["fp64"]) / torch.linalg.norm(sols["fp64"]))
        res["mixed"]["rel_error_vs_fp64_solution"] = err
        for name in ("fp64", "mixed"):
            res[name]["rel_error_vs_oracle_solution"] = float(torch.linalg.norm(sols[name] - U) / torch.linalg.norm(U))
        res["oracle_solution_s"] = oracle_s
        res["speedup_mixed_vs_fp64"] = res["fp64"]["ms"] / res["mixed"]["ms"]
        out[f"order{order}"] = res
        del sols, U
    return out


def run_batched(args):
    """Uneven batch: problems with sides 2^k + 1, k uniform in {7..11}, order 2 or 4
    (50/50), N(0,1) right-hand sides, mixed precision, each to 1e-8; the batched
    solve (hybrid schedule, and level-synchronous alone) vs the same problems solved
    one after another (median of three timed solves each)."""
    import numpy as np
    import torch
    import paper_2008_03885_gb300 as mg
    import synth
    count = args.batch_count
    z = synth.uniform01(SEED + 7, 2 * count)
    specs = [(2 ** (7 + int(z[2 * i] * 5)), 2 if z[2 * i + 1] < 0.5 else 4) for i in range(count)]
    rhs = {}
    for n, _ in specs:
        if n not in rhs:
            rhs[n] = torch.tensor(synth.rhs_normal(n, SEED + n), dtype=torch.float64, device="cuda")
    opts = dict(nu1=NU1, nu2=NU2, precision=mg.MG_PREC_MIXED_FP32, fma_contract=1, n_min=N_MIN_SMALL)
    t0 = time.perf_counter()
    hs = [mg.mg_setup(n, order, "redblack", "galerkin", **opts) for n, order in specs]
    fs = [rhs[n] for n, _ in specs]
    us = [torch.zeros_like(f) for f in fs]
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(solo_min_n):
        """Create the batch, warm it up (graph capture), then three timed solves from
        u = 0: the median time, the launches of one solve and the last cycles/residuals."""
        t0 = time.perf_counter()
        b = mg.mg_batch_create(hs, solo_min_n=solo_min_n)
        create_s = time.perf_counter() - t0
        mg.mg_batch_solve(b, us, fs, rtol=1e-8, max_cycles=40)
        times = []
        for _ in range(3):
            torch.cuda.synchronize()
            for u in us:
                u.zero_()
            l0 = mg.mg_batch_get_launches(b)
            e0.record(stream)
            cyc, rr = mg.mg_batch_solve(b, us, fs, rtol=1e-8, max_cycles=40)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            launches = mg.mg_batch_get_launches(b) - l0
        b.close()
        return sorted(times)[1], times, launches, cyc, rr, create_s

    # hybrid (library default: N >= 1024 solved alone on 12 worker streams) and the
    # level-synchronous schedule over every problem
    batch_ms, batch_times, batch_launches, cyc, rr, create_s = timed(0)
    sync_ms, sync_times, sync_launches, cyc_s, rr_s, _ = timed(1 << 20)
    # the same problems one after another through mg_solve (graphs warmed first)
    for h, u, f in zip(hs, us, fs):
        u.zero_()
        mg.mg_solve(h, u, f, rtol=1e-8, max_cycles=40)
    torch.cuda.synchronize()
    for u in us:
        u.zero_()
    e0.record(stream)
    for h, u, f in zip(hs, us, fs):
        mg.mg_solve(h, u, f, rtol=1e-8, max_cycles=40)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    for h in hs:
        h.close()
    points = sum((n - 1) ** 2 for n, _ in specs)
    return {"problems": count, "sides": "2^k+1, k uniform in {7..11}", "unknowns": points,
            "precision": "mixed FP32 inner / FP64 refinement", "rtol": 1e-8,
            "n_min": N_MIN_SMALL, "coarsest": f"dense solve of {(N_MIN_SMALL - 1) ** 2} unknowns",
            "schedule": "hybrid: N >= 1024 solved alone on 12 worker streams, the rest level-synchronous",
            "solo_problems": sum(1 for n, _ in specs if n >= 1024),
            "batch_ms": batch_ms, "batch_ms_runs": batch_times, "sequential_ms": seq_ms,
            "speedup": seq_ms / batch_ms, "max_cycles": max(cyc), "max_rel_res": max(rr),
            "batch_kernel_launches": batch_launches,
            "level_synchronous_ms": sync_ms, "level_synchronous_ms_runs": sync_times,
            "level_synchronous_launches": sync_launches, "level_synchronous_max_rel_res": max(rr_s),
            "unknowns_per_s": points / (batch_ms * 1e-3), "setup_s": setup_s, "batch_create_s": create_s}


def run_serving(args):
    """Seeded Poisson request stream at 2000 req/s, sides 2^k + 1 with k uniform in
    [8, 12], order 2/4 and Galerkin/non-Galerkin 50/50, tolerance 1e-8, 120 GB budget,
    one N(0,1) right-hand side per request (seeded by the request id, generated on the
    device when the request is taken up; every solution is copied back to host memory).
    Continuous batching (8 slots, mixed precision) serves the whole stream. The plain
    per-request FP64 solve (one slot, one request at a time) serves every
    `serve_plain_every`-th request of the same stream at the same arrival times, i.e. the
    offered rate divided by that factor: its capacity (~60 req/s) is far below 2000 req/s,
    so the whole stream would take over five minutes of one-at-a-time FP64 solves."""
    import torch
    from paper_2008_03885_gb300 import serve
    reqs = serve.poisson_stream(SEED, args.serve_count, 2000.0, 8, 12, rtol=1e-8, device_rhs=True)
    keys = sorted({(r.n, r.order, r.coarse_op) for r in reqs})
    out = {"requests": len(reqs), "rate_rps": 2000.0, "sides": "2^k+1, k uniform in [8, 12]",
           "rhs": "one N(0,1) field per request, seeded by the request id", "budget_gb": 120,
           "n_min": N_MIN_SMALL}
    plain = reqs[::args.serve_plain_every]
    for name, slots, opts, rq in (
            ("continuous_mixed", 8, dict(nu1=NU1, nu2=NU2, precision=1, fma_contract=1, n_min=N_MIN_SMALL), reqs),
            ("plain_fp64", 1, dict(nu1=NU1, nu2=NU2, n_min=N_MIN_SMALL), plain)):
        srv = serve.Server(slots=slots, budget_bytes=120e9, **opts)
        srv.warm(keys, per_key=min(slots, 2))
        results, stats = srv.run(rq, realtime=True, keep_u=False)
        srv.close()
        stats["max_rel_res"] = max(r.rel_res for r in results.values())
        stats["offered_rate_rps"] = 2000.0 * len(rq) / len(reqs)
        if rq is not reqs:
            stats["sample"] = (f"every {args.serve_plain_every}th request of the {len(reqs)}-request stream "
                               f"({len(rq)} requests) at their arrival times")
        out[name] = stats
        del results
        torch.cuda.empty_cache()
    return out


def run_profile_case(args):
    """A few finest-level kernels of the bench workload, for ncu captures: 4 smoothing
    sweeps, 2 residuals, 2 restrictions, 2 interpolations on level 0."""
    import torch
    import paper_2008_03885_gb300 as mg
    import synth
    n = args.profile_n
    F = synth.rhs_sine_modes(n, SEED)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    d = torch.zeros_like(f)
    h = mg.mg_setup(n, ORDER, "redblack", "galerkin", nu1=NU1, nu2=NU2)
    fc = mg.level_array(h, 1)
    for _ in range(2):
        mg.mg_level_smooth(h, 0, u, f, 2)
        mg.mg_level_residual(h, 0, u, f, d)
        mg.mg_level_restrict(h, 0, d, fc)
        mg.mg_level_prolong_add(h, 0, u, fc)
    torch.cuda.synchronize()
    h.close()
    print(json.dumps({"profile_case": n, "ok": True}))


def run_profile_solves(args, mixed: bool):
    """Two solves of the bench workload (warm-up + one), for ncu: mixed precision
    (FP32 inner cycles) or the FP64 headline solve. With --profile-batch-problem, three
    solves of one problem of the batch (N(0,1) right-hand side, n_min 16, to 1e-8)."""
    import torch
    import paper_2008_03885_gb300 as mg
    import synth
    n = args.profile_n
    batch = args.profile_batch_problem  # a problem of the batch: N(0,1), n_min 16, 1e-8
    rhs = synth.rhs_normal(n, 5) if batch else synth.rhs_sine_modes(n, SEED)
    f = torch.tensor(rhs, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    extra = dict(precision=mg.MG_PREC_MIXED_FP32, inner_cycles=1, fma_contract=1) if mixed else {}
    if batch:
        extra["n_min"] = N_MIN_SMALL
    h = mg.mg_setup(n, ORDER, "redblack", "galerkin", nu1=NU1, nu2=NU2, **extra)
    for _ in range(3 if batch else 2):
        u.zero_()
        k, hist = mg.mg_solve(h, u, f, rtol=1e-8 if batch else RTOL, max_cycles=60)
    torch.cuda.synchronize()
    h.close()
    print(json.dumps({"profile_mixed" if mixed else "profile_fp64": n, "cycles": k, "final": hist[-1]}))


# Algorithmic HBM bytes per fine grid point per cycle (every kernel reading its inputs
# and writing its outputs once; coarse levels of red-black coarsening add a factor
# sum 2^-l = 2): FP64 V(2,1) 224 B, FP32 V(2,1) 112 B; a refinement step adds the FP64
# residual (read u, f: 16 B; write the FP32 copy: 4 B) and the update (read u, e; write
# u: 20 B) to the FP32 cycle.
BYTES_PER_POINT_FP64_V21 = 224
BYTES_PER_POINT_MIXED_STEP = 20 + 112 + 20


def solve_throughput(fp64_ms, fp64_cycles, mixed):
    """Grid-point-cycles/s and effective HBM GB/s of whole solves, FP64 vs mixed."""
    pts = (N + 1) ** 2
    out = {"fp64": {"grid_point_cycles_per_s": pts * fp64_cycles / (fp64_ms * 1e-3),
                    "effective_hbm_gbs": BYTES_PER_POINT_FP64_V21 * pts * fp64_cycles / (fp64_ms * 1e-3) / 1e9}}
    if mixed:
        out["mixed"] = {"grid_point_cycles_per_s": pts * mixed["cycles"] / (mixed["ms"] * 1e-3),
                        "effective_hbm_gbs": BYTES_PER_POINT_MIXED_STEP * pts * mixed["cycles"]
                        / (mixed["ms"] * 1e-3) / 1e9}
    out["model"] = ("algorithmic bytes per fine point per cycle: FP64 V(2,1) 224 (both FP64-pipe and "
                    "latency bound, so far below HBM); mixed refinement step 152 (FP64 residual 20 + "
                    "FP32 V(2,1) 112 + FP64 update 20)")
    return out


def run_fp_pipe_probe():
    """Compile FP_PIPE_PROBE_CU for sm_103a and run it (prints G operations/s per kind)."""
    from paper_2008_03885_gb300 import _build
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "fp_pipe_probe.cu"), os.path.join(d, "fp_pipe_probe")
        with open(src, "w") as fh:
            fh.write(FP_PIPE_PROBE_CU)
        subprocess.run([_build.nvcc(), *_build.ARCH, "-O3", "-o", exe, src], check=True)
        subprocess.run([exe], check=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-n", type=int, default=N, help="grid of the reference arm (the oracle)")
    ap.add_argument("--no-all-cores", action="store_true", help="reference arm: skip the all-cores run")
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", action="store_true", help="run a few finest-level kernels (ncu)")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and serving measurements")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--large-n", type=int, default=8192)
    ap.add_argument("--serve-count", type=int, default=20000)
    ap.add_argument("--serve-plain-every", type=int, default=10)
    ap.add_argument("--profile-n", type=int, default=4096)
    ap.add_argument("--profile-batch-problem", action="store_true",
                    help="profile solves: the batch's settings (N(0,1) right-hand side, n_min 16, 1e-8; three solves)")
    ap.add_argument("--profile-mixed", action="store_true", help="two mixed-precision solves (ncu)")
    ap.add_argument("--profile-fp64", action="store_true", help="two FP64 solves of the bench workload (ncu)")
    ap.add_argument("--fp-pipe-probe", action="store_true", help="FP64/FP32 arithmetic issue rates (microbenchmark)")
    args = ap.parse_args()
    if args.fp_pipe_probe:
        run_fp_pipe_probe()
        return
    if args.profile_case:
        run_profile_case(args)
        return
    if args.profile_mixed or args.profile_fp64:
        run_profile_solves(args, mixed=args.profile_mixed)
        return
    ws, rank, local = dist_env()
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
