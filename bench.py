#!/usr/bin/env python
"""Benchmark: LQ-MPC interior-point solves/s and per-iteration KKT time at a
1e-8 scaled KKT residual, mixed precision (tensor-core formation of M, FP32
Cholesky, FP64 refinement and fallback; --precision picks the formation:
split TF32 = FP32-accurate (default), BF16 or TF32) versus FP64, on the 2-D
heat plant of a 32 x 32 grid (ns = 1024, nu = 10, N = 50; M is 500 x 500).

One step = one full IPM solve (all per-iteration steps of the hot path) for
one seeded initial state x0.  Inputs sit in device memory before the timed
region; L2 is flushed (512 MB write) between steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs are independent replicas (one process per GPU, disjoint x0
seeds, no collective in the data path): value = all solves / max-over-ranks
time.  The reference arm is the CPU oracle (FP64 Riccati-Mehrotra), timed on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2209_13049_b300 import inputs  # noqa: E402

METRIC = "LQ-MPC IPM solves/s & per-iter KKT ms at 1e-8 residual, mixed vs FP64"
WORKLOAD = "heat2d 32x32 (ns=1024, nu=10, N=50), x0 = seeded 8-Gaussian fields, tol 1e-8"
GOLD = os.path.join(ROOT, "tests", "golden", "heat2d_g32_nu10_N50.npz")
NS, NU, N = 1024, 10, 50
# DRAM bytes (read + write) of one k_potrf_flow launch on this workload from the
# ncu capture summarised in profiles/ (None until captured for this kernel version)
POTRF_FLOW_TRAFFIC = 765696
DTYPES = {
    "fp32": "mixed: FP32-accurate formation on tcgen05 (split TF32, FP32 accumulate), FP32 Cholesky, two-level "
            "FP32 tier near the end, FP64-accurate refinement, FP64 fallback",
    "bf16": "mixed: BF16 tcgen05 formation (FP32 accumulate), FP32 Cholesky, two-level FP32 tier, FP64-accurate "
            "refinement, FP64 fallback",
    "tf32": "mixed: TF32 tcgen05 formation (FP32 accumulate), FP32 Cholesky, two-level FP32 tier, FP64-accurate "
            "refinement, FP64 fallback",
    "fp64": "f64",
}


def syrk_alg_flops(ns, nu, N):
    """Algorithmic flops of one KKT-matrix formation exploiting the block
    lower-triangular Toeplitz structure of Gamma: the lower-triangle blocks
    (j >= k) each need N - j products G_p' D G_q of 2 ns nu^2 flops."""
    return 2.0 * ns * nu * nu * N * (N + 1) * (N + 2) / 6.0


def lyap_fma(p):
    """Multiply-adds of the FP64 Horner-chain formation of M for plant p: per
    (block column c, input col) N sparse products A'z, N-c scaled G-stack
    columns and c+1 sparse dots with B's columns."""
    import scipy.sparse as sp
    nnz_a = sp.csr_matrix(p.A).nnz
    nnz_b = int(np.count_nonzero(p.B))
    return p.N * p.N * p.nu * float(nnz_a) + 0.5 * p.N * (p.N + 1) * p.nu * float(p.ns + nnz_b)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_baseline(seconds_budget: float = 30.0):
    """The oracle as it stands, single-threaded, on one full solve of the
    workload (seed 0): about 25 s on one host core."""
    import oracle
    plant, x0 = inputs.config_2d_32(0)
    t = time.perf_counter()
    r = oracle.ipm_solve(plant, x0, tol=1e-8)
    dt = time.perf_counter() - t
    return {"value": 1.0 / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"1 full solve (x0 seed 0, {r['stats']['iters']} iterations) of the workload, "
                      f"{dt:.1f} s on 1 host core ({len(os.sched_getaffinity(0))} available)"}


def run_reference(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    import oracle
    plant, x0s = inputs.heat2d(32, 10, 50), None
    full_iters = None
    if os.path.exists(GOLD):
        full_iters = len(np.load(GOLD)["heat2d_32_s0_trace8"]) - 1
    per_iter = []
    sample_iters = 2
    for step in range(args.warmup + args.steps):
        x0 = inputs.x0_gaussians(32, step)
        t = time.perf_counter()
        r = oracle.ipm_solve(plant, x0, tol=1e-8, max_iter=sample_iters)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            per_iter.append(dt / max(1, r["stats"]["iters"]))
    if full_iters is None:
        full_iters = oracle.ipm_solve(plant, inputs.x0_gaussians(32, 0), tol=1e-8)["stats"]["iters"]
    t_iter = float(np.mean(per_iter))
    value = 1.0 / (t_iter * full_iters)
    ms_per_step = t_iter * sample_iters * 1e3
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "ns": NS, "nu": NU, "N": N},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: {sample_iters} IPM iterations of the oracle on one x0; "
                                       f"solves/s = 1/(time per iteration x {full_iters} iterations of a full "
                                       f"solve of x0 seed 0)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2209_13049_b300 import binding, build
    build.build()
    binding.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    plant = inputs.heat2d(32, 10, 50)
    K, W = args.steps, args.warmup
    seeds = [rank * 100000 + i for i in range(W + K)]
    x0_host = [inputs.x0_gaussians(32, s) for s in seeds]
    x0_dev = [torch.tensor(x, dtype=torch.float64, device=dev) for x in x0_host]
    u_dev = [torch.zeros(plant.n, dtype=torch.float64, device=dev) for _ in seeds]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed_solves(solver, idx, use_host=False):
        """Per-step CUDA-event times (ms) on the solver's stream; L2 flushed between steps."""
        times, stats = [], []
        for i in idx:
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if use_host:
                u, st = solver.solve(x0_host[i], check=False)
            else:
                st = solver.solve_device(x0_dev[i], u_dev[i], check=False)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            stats.append(st)
        return times, stats

    mixed = binding.Solver(plant, precision=args.precision, stream=stream)
    fp64 = binding.Solver(plant, precision="fp64", stream=stream)

    # warm-up
    timed_solves(mixed, range(W))
    timed_solves(fp64, range(min(W, 1)))
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = binding.kernel_launches()
    barrier()
    torch.cuda.nvtx.range_push("timed")
    t_mixed, st_mixed = timed_solves(mixed, range(W, W + K))
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = binding.kernel_launches() - launches0
    clocks = sampler.stop()
    # FP64 comparison (fewer steps: each FP64 solve is ~10x longer)
    kf = max(1, min(K, args.fp64_steps))
    t_fp64, st_fp64 = timed_solves(fp64, range(W, W + kf))
    # end-to-end through the host API (x0 from host, u back to host, inside the call)
    t_e2e, _ = timed_solves(mixed, range(W, W + K), use_host=True)
    barrier()

    total_ms = float(sum(t_mixed))
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([total_ms, float(sum(t_e2e))], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms, e2e_ms = float(tt[0]), float(tt[1])
    else:
        e2e_ms = float(sum(t_e2e))
    value = world * K / (total_ms / 1e3)
    e2e_value = world * K / (e2e_ms / 1e3)

    # parity against the stored oracle results for x0 seed 0: at the same stop
    # tolerance (1e-8, "u8") and against the tight optimum (1e-12, "u12")
    errs = {}
    if os.path.exists(GOLD):
        g = np.load(GOLD)
        x0g = g["heat2d_32_s0_x0"]
        u_m, _ = mixed.solve(x0g, check=False)
        u_f, _ = fp64.solve(x0g, check=False)
        for key in ("u8", "u12"):
            ref = g[f"heat2d_32_s0_{key}"]
            scale = max(1.0, float(np.max(np.abs(ref))))
            errs[f"mixed_vs_oracle_{key}"] = float(np.max(np.abs(u_m - ref)) / scale)
            errs[f"fp64_vs_oracle_{key}"] = float(np.max(np.abs(u_f - ref)) / scale)

    def summary(times, stats):
        iters = [s["iters"] for s in stats]
        kkt = [s["t_kkt_ms"] / max(1, s["iters"]) for s in stats]
        return {"solves_per_s": len(times) / (sum(times) / 1e3), "ms_per_solve": float(np.mean(times)),
                "iters_mean": float(np.mean(iters)), "kkt_ms_per_iter": float(np.mean(kkt)),
                "refine_steps_mean": float(np.mean([s["refine_steps"] for s in stats])),
                "fallbacks_total": int(sum(s["fallbacks"] for s in stats)),
                "status": sorted({int(s["status"]) for s in stats})}

    # Rooflines from the library's CUDA events around the launches inside the
    # timed solves.  The dominant kernel of a mixed solve (ncu launch list in
    # profiles/) is the FP32 Cholesky with the inverse (k_potrf_flow, one
    # instance): latency-bound, so it is reported against the FP32 FMA pipe
    # (148 SMs x 128 FMA/clk x 2 flop x SM clock); algorithmic work = n^3/3
    # (factor) + n^3/3 (triangular inverse).  Beside it: the tensor-core
    # formation of M and the FP64 formation.
    peaks, which = measured_peaks()
    sm_mhz = clocks.get("sm_mhz") or 2032.0
    n = NU * N
    npf = sum(s["potrf32_launches"] for s in st_mixed)
    tpf = sum(s["t_potrf32_ms"] for s in st_mixed)
    pf_flops = 2.0 * n ** 3 / 3.0
    fp32_peak = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12
    ach_pf = pf_flops / (tpf / max(1, npf) / 1e3) / 1e12 if npf else None
    roofline = {"kernel": "k_potrf_flow (FP32 Cholesky + inverse of the factor, n = 500)", "bound": "alu",
                "achieved": ach_pf, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": (ach_pf / fp32_peak) if ach_pf else None, "traffic": POTRF_FLOW_TRAFFIC,
                "peak_source": f"derived: 148 SMs x 128 FP32 FMA/clk x 2 flop x {sm_mhz:.0f} MHz (median SM clock "
                               f"sampled during the timed region); latency-bound (one diagonal block after another)",
                "flops_per_launch": pf_flops, "launches": npf,
                "avg_launch_us": (tpf / max(1, npf) * 1e3) if npf else None}
    flops = syrk_alg_flops(NS, NU, N)
    n3 = sum(s["syrk_tc3_launches"] for s in st_mixed)
    t3 = sum(s["t_syrk_tc3_ms"] for s in st_mixed)
    n1 = sum(s["syrk_tc_launches"] for s in st_mixed) - n3
    t1 = sum(s["t_syrk_tc_ms"] for s in st_mixed) - t3
    tf32_peak = peaks.get("bf16_tflops_sustained", 1400.0) * 0.5      # nominal TF32 : BF16 = 1 : 2
    bf16_peak = peaks.get("bf16_tflops_sustained", 1400.0)
    roofline_tc = {
        "kernel": "k_syrk_tc (tcgen05 formation of M, Eq. 7)", "bound": "tensor", "unit": "TFLOP/s",
        "algorithmic_flops_per_launch": flops,
        "split_tf32": {"launches": n3, "avg_launch_us": (t3 / n3 * 1e3) if n3 else None,
                       "executed_flops_per_launch": 3 * flops,
                       "achieved": (3 * flops / (t3 / n3 / 1e3) / 1e12) if n3 else None, "peak": tf32_peak,
                       "frac": (3 * flops / (t3 / n3 / 1e3) / 1e12 / tf32_peak) if n3 else None,
                       "peak_source": f"{which} bf16_tflops_sustained x 0.5 (nominal TF32 rate)"},
        "bf16": {"launches": n1, "avg_launch_us": (t1 / n1 * 1e3) if n1 else None,
                 "achieved": (flops / (t1 / n1 / 1e3) / 1e12) if n1 else None, "peak": bf16_peak,
                 "frac": (flops / (t1 / n1 / 1e3) / 1e12 / bf16_peak) if n1 else None,
                 "peak_source": f"{which} bf16_tflops_sustained"}}
    n64 = sum(s["syrk_fp64_launches"] for s in st_fp64)
    t64 = sum(s["t_syrk_fp64_ms"] for s in st_fp64)
    fp64_peak = 148 * 2 * 2 * sm_mhz * 1e6 / 1e12
    ly_flops = 2.0 * lyap_fma(plant)
    roofline_fp64 = {"kernel": "FP64 formation of M by Horner chains over the horizon (k_ly_chain)", "bound": "alu",
                     "unit": "TFLOP/s", "launches": n64, "avg_us": (t64 / n64 * 1e3) if n64 else None,
                     "algorithmic_flops": ly_flops,
                     "achieved": (ly_flops / (t64 / n64 / 1e3) / 1e12) if n64 else None, "peak": fp64_peak,
                     "frac": (ly_flops / (t64 / n64 / 1e3) / 1e12 / fp64_peak) if n64 else None,
                     "peak_source": "derived: 148 SMs x 2 FP64 FMA/clk x 2 flop x SM clock"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPES[args.precision],
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "ns": NS, "nu": NU, "N": N,
                           "l2": "flushed between steps (512 MB write, outside the timed events)",
                           "parallelism": f"replicas x{world}", "precision": args.precision},
                "mixed": summary(t_mixed, st_mixed), "fp64": summary(t_fp64, st_fp64),
                "speedup_mixed_vs_fp64": (value / world) / (kf / (sum(t_fp64) / 1e3)),
                "u_rel_err_vs_oracle": errs, "roofline": roofline, "roofline_tensor_syrk": roofline_tc,
                "roofline_fp64_formation": roofline_fp64,
                "clocks": clocks,
                "gpu_launches": int(launches),
                "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": NS * 8,
                        "d2h_bytes_per_step": plant.n * 8}}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_baseline()
        print(json.dumps(line), flush=True)
    mixed.close()
    fp64.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batch(args):
    """Uneven batch of 256 instances (1-D or 2-D heat plants, ns 200-2000,
    nu 2-16, N 10-50) solved in lockstep through lqmpc_solve_batch: host x0 in,
    host u out, copies inside the timed call."""
    import torch
    from paper_2209_13049_b300 import binding, build
    torch.cuda.set_device(0)
    build.build()
    binding.load()
    inst = inputs.batch_instances(args.batch, 0)
    t0 = time.perf_counter()
    solvers = [binding.Solver(p, precision=args.precision) for p, _ in inst]
    t_setup = time.perf_counter() - t0
    x0s = [x for _, x in inst]
    t0 = time.perf_counter()
    binding.autotune(solvers)       # launch shapes for this batch signature (measured)
    t_tune = time.perf_counter() - t0
    for _ in range(args.warmup):
        binding.solve_batch(solvers, x0s, check=False)
    times, launches = [], []
    sampler = ClockSampler(0)
    sampler.start()
    for _ in range(args.steps):
        k0 = binding.kernel_launches()
        torch.cuda.synchronize()
        t = time.perf_counter()
        us, stats, code = binding.solve_batch(solvers, x0s, check=False)
        times.append(time.perf_counter() - t)
        launches.append(binding.kernel_launches() - k0)
    clocks = sampler.stop()
    # parity: batched lockstep result against each sampled instance solved alone in FP64
    errs = []
    for k in range(0, len(inst), max(1, len(inst) // 8)):
        ref, _ = binding.Solver(inst[k][0], precision="fp64").solve(x0s[k], check=False)
        errs.append(float(np.max(np.abs(us[k] - ref)) / max(1.0, float(np.max(np.abs(ref))))))
    ms = 1e3 * float(np.mean(times))
    n = [p.n for p, _ in inst]
    line = {"metric": "uneven-batch LQ-MPC IPM solves/s at 1e-8 residual", "value": len(inst) / (ms / 1e3),
            "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "data": "synthetic",
            "config": {"workload": f"{len(inst)} instances, coin-flip heat1d (ns 200-2000) / heat2d (g 15-44), "
                                   f"nu 2-16, N 10-50 (n {min(n)}-{max(n)}), master seed 0",
                       "api": "lqmpc_solve_batch (host buffers, copies inside the call)"},
            "iters_max": int(max(s["iters"] for s in stats)), "status": sorted({int(s["status"]) for s in stats}),
            "fallbacks_total": int(sum(s["fallbacks"] for s in stats)), "gpu_launches": int(np.mean(launches)),
            "setup_s": t_setup, "autotune_s": t_tune, "u_rel_err_vs_single_fp64_max": max(errs), "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_warmstart(args):
    """Learned warm start on the heat2d 32x32 plant: (x0, u*) pairs from
    lockstep batches of the GPU solver, the 1024 -> 512 -> 512 -> 500 network
    trained by the library's own kernels, then warm- versus cold-started
    solves on held-out x0 (seeds 10^6 + k)."""
    import torch
    from paper_2209_13049_b300 import binding, build
    torch.cuda.set_device(0)
    build.build()
    binding.load()
    plant = inputs.heat2d(32, 10, 50)
    S, H, E = args.train_pairs, args.heldout, args.epochs
    solvers = [binding.Solver(plant, precision=args.precision) for _ in range(256)]
    t0 = time.perf_counter()
    xs, us = [], []
    for k0 in range(0, S, 256):
        x0s = [inputs.x0_gaussians(32, s) for s in range(k0, min(S, k0 + 256))]
        u, st, code = binding.solve_batch(solvers[:len(x0s)], x0s, check=False)
        xs += x0s
        us += u
    t_data = time.perf_counter() - t0
    X, U = np.array(xs), np.array(us)
    net = binding.MLP(plant.ns, 512, plant.n, max_batch=256, seed=1)
    net.set_bounds(np.tile(plant.ul, plant.N), np.tile(plant.uu, plant.N))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.train(X, U, epochs=E, batch=256, lr=args.lr, seed=2)
    t_train = time.perf_counter() - t0
    xt = np.array([inputs.x0_gaussians(32, 10**6 + k) for k in range(H)])
    t0 = time.perf_counter()
    guess = net.infer(xt)
    t_infer = time.perf_counter() - t0
    s = solvers[0]
    cold_t, warm_t, cold_it, warm_it, errs = [], [], [], [], []
    for k in range(H):
        t = time.perf_counter()
        uc, stc = s.solve(xt[k], check=False)
        cold_t.append(time.perf_counter() - t)
        t = time.perf_counter()
        uw, stw = s.solve_warm(xt[k], guess[k], check=False)
        warm_t.append(time.perf_counter() - t)
        cold_it.append(stc["iters"])
        warm_it.append(stw["iters"])
        errs.append(float(np.max(np.abs(uw - uc)) / max(1.0, float(np.max(np.abs(uc))))))
    steps = E * (S // 256)
    line = {"metric": "warm- vs cold-started LQ-MPC IPM solves/s at 1e-8 residual", "unit": "solves/s",
            "value": H / sum(warm_t), "cold_value": H / sum(cold_t), "n_gpus": 1, "higher_is_better": True,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"heat2d 32x32 (ns=1024, nu=10, N=50); MLP 1024-512-512-500 BF16; "
                                   f"{S} training pairs (x0 seeds 0..{S - 1}), {H} held-out (seeds 1e6..)",
                       "train": {"epochs": E, "batch": 256, "lr": args.lr}},
            "iters_cold_mean": float(np.mean(cold_it)), "iters_warm_mean": float(np.mean(warm_it)),
            "ms_cold_mean": 1e3 * float(np.mean(cold_t)), "ms_warm_mean": 1e3 * float(np.mean(warm_t)),
            "u_rel_err_warm_vs_cold_max": max(errs), "data_gen_s": t_data,
            "train_s": t_train, "train_samples_per_s": steps * 256 / t_train,
            "loss_first_last": [float(losses[0]), float(losses[-1])], "infer_ms": 1e3 * t_infer}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["bf16", "tf32", "fp32", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="heat2d32", choices=["heat2d32", "batch", "warmstart"],
                    help="heat2d32: the metric's workload; batch: the uneven lockstep batch; "
                         "warmstart: the learned warm start")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--train-pairs", type=int, default=4096)
    ap.add_argument("--heldout", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--lr", type=float, default=1e-3)
    args = ap.parse_args()
    if args.workload == "batch":
        run_batch(args)
    elif args.workload == "warmstart":
        run_warmstart(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
