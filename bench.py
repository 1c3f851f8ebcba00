#!/usr/bin/env python3
"""Benchmark of the RFPF Cholesky hot path on GB300.

One step = one pass of the whole path over one synthetic SPD matrix held in
one of the eight RFPF layouts: step s uses TRANSR x UPLO pair s mod 4 and
order n = 16384 (even) for (s div 4) even, n = 16383 (odd, the leading
principal submatrix) otherwise, so 8 steps cover all eight layouts:
  rfp_dpack (full -> RFPF), rfp_dpftrf, rfp_dpftrs (nrhs = 256),
  rfp_dpftri, rfp_dunpack (RFPF -> full, the inverse).
A = Q diag(lam) Q^T, Q Haar-random orthogonal, lam log-uniform on [1, 1e4]
(rfp_inputs.spd_spectrum, seed 0); B uniform[-1, 1].  Inputs are resident in
HBM before the timed region and larger than L2 (the RFP array alone is
1.07 GB), so no L2 flush is needed.

Reported metric: PFTRF+PFTRS TFLOP/s = (n^3/3 + 2 n^2 nrhs)
summed over the timed steps / the device time of those two calls (CUDA
events on the launching stream).  The other rows of the step are reported in
"breakdown".  --impl reference times the plain CPU oracle on the host cores
instead (a bounded sample of the same workload per step).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# dram__bytes_read.sum + dram__bytes_write.sum of the PFTRF step-3 launch at
# n = 16384 (one ncu capture of the unchanged kernel, summarized under
# profiles/): 6.38 GB + 0.276 GB.
SYRK_TRAFFIC_N16384 = 6.656e9
METRIC = "PFTRF+PFTRS TFLOP/s & % peak; served solves/s, p50/p99 at ≤1e-12 bwd err"
LAYOUTS = [(t, u) for t in "NT" for u in "LU"]


def step_layout(s: int, n: int):
    """(transr, uplo, order) of step s: 4 TRANSR x UPLO pairs x 2 parities."""
    transr, uplo = LAYOUTS[s % 4]
    return transr, uplo, (n if (s // 4) % 2 == 0 else n - 1)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=8)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--nrhs", type=int, default=256)
    p.add_argument("--kappa", type=float, default=1e4)
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--cpu-n", type=int, default=0,
                   help="oracle sample order (default 10240 for cpu_baseline, 6144 per "
                        "reference step)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--mode", choices=["fp64", "mixed", "batched", "serve", "surface", "c1"],
                   default="fp64",
                   help="fp64: the FP64 hot path (default line); mixed: the mixed-precision "
                        "solve at n = 32768 against the FP64 path (its own line)")
    p.add_argument("--mixed-n", type=int, default=32768)
    p.add_argument("--mixed-nrhs", type=int, default=64)
    p.add_argument("--kappas", default="1e2,1e4,1e6")
    p.add_argument("--precs", default="fp32,tf32x3,bf16x6,tf32,bf16")
    p.add_argument("--max-iter", type=int, default=30, help="refinement steps (mixed mode)")
    p.add_argument("--batch", type=int, default=4096, help="batched mode: matrices per batch")
    p.add_argument("--serve-requests", type=int, default=1000,
                   help="serve mode: requests per run (the stream description uses 20000)")
    p.add_argument("--serve-pool", type=int, default=64, help="serve mode: distinct matrices")
    p.add_argument("--serve-loads", default="0.5,0.7,0.9",
                   help="serve mode: offered loads as fractions of the measured capacity")
    p.add_argument("--retune", action="store_true",
                   help="batched mode: re-run the panel-width autotuner even if cached")
    p.add_argument("--no-fp64-ref", action="store_true",
                   help="mixed mode: skip the FP64 PFTRF + PFTRS reference run")
    p.add_argument("--legs", default="c1,mixed,batched,serve",
                   help="fp64 mode at N = 1: the other configurations measured after the main "
                        "timed region and reported under breakdown (empty: none)")
    return p.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sms = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sms)}


# ---------------------------------------------------------------------------
# CPU oracle legs (cpu_baseline and --impl reference)

def oracle_sample(n: int, nrhs: int, kappa: float, seed: int = 0):
    """Time the plain oracle's PFTRF + PFTRS on an n x n matrix of the same
    recipe; returns (TFLOP/s, seconds, threads)."""
    import numpy as np

    import oracle
    import rfp_inputs as gen
    from paper_0901_1696_gb300.flops import pftrf_flops, pftrs_flops
    A = gen.spd_spectrum(n, seed=seed, kappa=kappa)
    B = gen.rhs(n, nrhs, seed=seed + 1)
    arf = oracle.pack("N", "L", A)
    t0 = time.perf_counter()
    fac, info = oracle.pftrf("N", "L", n, arf)
    oracle.pftrs("N", "L", n, fac, B)
    dt = time.perf_counter() - t0
    assert info == 0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return (pftrf_flops(n) + pftrs_flops(n, nrhs)) / dt / 1e12, dt, threads


def run_reference(args, rank: int):
    if rank != 0:
        return
    args.cpu_n = args.cpu_n or 6144
    nrhs = max(1, args.nrhs * args.cpu_n // args.n)
    times, rates = [], []
    for s in range(args.warmup + args.steps):
        rate, dt, threads = oracle_sample(args.cpu_n, nrhs, args.kappa, seed=s)
        if s >= args.warmup:
            times.append(dt)
            rates.append(rate)
    total_flops = len(times) * ((args.cpu_n ** 3) / 3 + 2 * args.cpu_n ** 2 * nrhs)
    value = total_flops / sum(times) / 1e12
    sample = (f"plain C oracle PFTRF+PFTRS (unpack, textbook Cholesky, substitution), "
              f"n={args.cpu_n}, nrhs={nrhs}, layout N/L, same spectrum recipe (kappa="
              f"{args.kappa:g}), one matrix per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"FP64 SPD RFPF PFTRF+PFTRS, oracle sample n={args.cpu_n} "
                               f"(of n={args.n}), nrhs={nrhs}", "kappa": args.kappa},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU leg

def fp64_peak_tflops(sm_mhz: float | None) -> float:
    """FP64 FMA peak of GB300 from unit counts and clock: 152 SMs x
    FP64_FMA_PER_SM_CLK FMAs x 2 flops x SM clock (MHz)."""
    from paper_0901_1696_gb300.peaks import FP64_FMA_PER_SM_CLK, SM_COUNT, SM_MAX_MHZ
    mhz = sm_mhz or SM_MAX_MHZ
    return SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12


def replica_max(dist, device, *ms):
    """Each time (ms) maximised over the ranks of the process group (the
    slowest replica bounds the job); the times unchanged without one."""
    if dist is None:
        return [float(x) for x in ms]
    import torch
    t = torch.tensor([float(x) for x in ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def replica_value(world: int, flops_per_rank: float, max_ms: float) -> float:
    """Whole-job rate (TFLOP/s): every replica did flops_per_rank within max_ms."""
    return world * flops_per_rank / (max_ms * 1e-3) / 1e12


def run_ours(args, rank: int, world: int):
    import numpy as np
    import torch

    import rfp_inputs as gen
    from paper_0901_1696_gb300 import binding as rfp
    from paper_0901_1696_gb300.flops import pack_bytes, pftrf_flops, pftri_flops, pftrs_flops

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    lib = rfp.library()
    n, nrhs = args.n, args.nrhs
    nt = n * (n + 1) // 2

    A = gen.spd_spectrum(n, seed=0, kappa=args.kappa, device=dev)     # symmetric: col-major
    Bh = gen.rhs(n, nrhs, seed=1)
    B0 = torch.from_numpy(np.ascontiguousarray(Bh.T)).to(dev)          # (nrhs, n) = col-major
    X = torch.empty_like(B0)
    arf = torch.empty(nt, dtype=torch.float64, device=dev)
    Ainv = torch.zeros(n, n, dtype=torch.float64, device=dev)
    infos = torch.zeros(args.warmup + args.steps, 2, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rows = ["pack", "pftrf", "pftrs", "pftri", "unpack"]

    def step(s, evs=None):
        transr, uplo, m = step_layout(s, n)      # A(0:m, 0:m), leading dimension n
        rec = (lambda i: evs[i].record(stream)) if evs else (lambda i: None)
        rec(0)
        lib.rfp_dpack(transr, uplo, m, A, n, arf, stream)
        rec(1)
        lib.rfp_dpftrf(transr, uplo, m, arf, infos[s, 0:1], stream)
        rec(2)
        X.copy_(B0)
        rec(3)
        lib.rfp_dpftrs(transr, uplo, m, nrhs, arf, X, n, stream)
        rec(4)
        lib.rfp_dpftri(transr, uplo, m, arf, infos[s, 1:2], stream)
        rec(5)
        lib.rfp_dunpack(transr, uplo, m, arf, Ainv, n, stream)
        rec(6)

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize(dev)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(args.steps)]
    t_begin, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = lib.rfp_kernel_launches()
    lib.rfp_stage_timing(True)
    sampler.start()
    t_begin.record(stream)
    for k in range(args.steps):
        step(args.warmup + k, evs[k])
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    stages = lib.rfp_stage_times()
    lib.rfp_stage_timing(False)
    launches = lib.rfp_kernel_launches() - launches0
    if dist:
        dist.barrier()
    total_ms = t_begin.elapsed_time(t_end)
    assert int(infos.abs().sum().item()) == 0, "a factorization reported info != 0"

    per_row = {r: 0.0 for r in rows}
    for ev in evs:
        per_row["pack"] += ev[0].elapsed_time(ev[1])
        per_row["pftrf"] += ev[1].elapsed_time(ev[2])
        per_row["pftrs"] += ev[3].elapsed_time(ev[4])
        per_row["pftri"] += ev[4].elapsed_time(ev[5])
        per_row["unpack"] += ev[5].elapsed_time(ev[6])
    K = args.steps
    orders = [step_layout(args.warmup + k, n)[2] for k in range(K)]
    metric_ms = per_row["pftrf"] + per_row["pftrs"]
    metric_flops = sum(pftrf_flops(m) + pftrs_flops(m, nrhs) for m in orders)
    metric_ms, total_ms = replica_max(dist, dev, metric_ms, total_ms)
    value = replica_value(world, metric_flops, metric_ms)

    # steps of the paper's Fig. 4 (PFTRF) and the dominant kernel's launch:
    # step 3 (T2 -= S S^T) is a single gemm_nt_kernel<double> launch
    agg = {}
    for name, ms in stages:
        agg[name] = agg.get(name, 0.0) + ms
    # algorithmic flops of step 3 (lower triangle of T2 incl. its diagonal:
    # n2 (n2 + 1) / 2 dot products of length n1, 2 flops each) per step
    syrk_ms = agg.get("pftrf.syrk_t2", 0.0) / K
    syrk_flops = 0.0
    for k, m in enumerate(orders):
        uplo = step_layout(args.warmup + k, n)[1]
        n1 = (m + 1) // 2 if uplo == "L" else m // 2
        syrk_flops += n1 * (m - n1) * (m - n1 + 1) / K
    peak = fp64_peak_tflops(clocks["sm_mhz"])
    achieved = syrk_flops / (syrk_ms * 1e-3) / 1e12 if syrk_ms else None
    pf = [agg.get(k, 0.0) for k in ("pftrf.potrf_t1", "pftrf.trsm_s", "pftrf.syrk_t2",
                                    "pftrf.potrf_t2")]
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"FP64 SPD n={n}/{n - 1} RFPF, all 8 layouts cycled over the steps; "
                               f"pack + PFTRF + PFTRS(nrhs={nrhs}) + PFTRI + unpack",
                   "n": [n, n - 1], "nrhs": nrhs,
                   "kappa": args.kappa, "matrix": "Q diag(lam) Q^T, Haar Q, log-uniform lam",
                   "l2": "inputs larger than L2 (RFP 1.07 GB); no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": SYRK_TRAFFIC_N16384 if n == 16384 else None,
                     "traffic_source": "profiles/gemm_nt_syrk_n16384_traffic.md (ncu, one launch "
                                       "at n = 16384)" if n == 16384 else None,
                     "kernel": "gemm_nt_kernel<double>: PFTRF step 3 (T2 -= S S^T), one launch",
                     "peak_source": "FP64 FMA pipe: 152 SMs x units x 2 x median SM clock"},
        "breakdown": {
            **{f"{r}_ms": per_row[r] / K for r in rows},
            "pftrf_tflops": sum(map(pftrf_flops, orders)) / (per_row["pftrf"] * 1e-3) / 1e12,
            "pftrs_tflops": sum(pftrs_flops(m, nrhs) for m in orders) / (per_row["pftrs"] * 1e-3) / 1e12,
            "pftri_tflops": sum(map(pftri_flops, orders)) / (per_row["pftri"] * 1e-3) / 1e12,
            "pack_gbs": sum(map(pack_bytes, orders)) / (per_row["pack"] * 1e-3) / 1e9,
            "unpack_gbs": sum(map(pack_bytes, orders)) / (per_row["unpack"] * 1e-3) / 1e9,
            "pftrf_step_split": [round(x / sum(pf), 4) for x in pf] if sum(pf) else None,
            "pftri_steps_ms": {k: v / K for k, v in agg.items() if k.startswith("pftri.")},
        },
        "clocks": clocks,
        "gpu_launches": launches,
    }

    if not args.no_e2e:
        e2e = e2e_leg(args, lib, A, B0, dev, stream)
        e2e_ms, = replica_max(dist, dev, e2e["ms_per_step"])
        e2e["ms_per_step"] = e2e_ms
        e2e["value"] = replica_value(world, pftrf_flops(n) + pftrs_flops(n, nrhs), e2e_ms)
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline:
        args.cpu_n = args.cpu_n or 10240
        rate, dt, threads = oracle_sample(args.cpu_n, max(1, nrhs * args.cpu_n // n), args.kappa)
        line["config"]["cpu_baseline_sample"] = (
            f"oracle timed on a smaller sample of the same recipe: n={args.cpu_n}, nrhs="
            f"{max(1, nrhs * args.cpu_n // n)} (the oracle's rate is roughly flat in n; n={n} "
            "would take about a minute of host time)")
        line["cpu_baseline"] = {
            "value": rate, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"plain C oracle PFTRF+PFTRS at n={args.cpu_n}, nrhs="
                      f"{max(1, nrhs * args.cpu_n // n)}, layout N/L, same recipe ({dt:.1f} s)"}
    if world == 1 and args.legs:
        del A, Ainv, arf, X, B0
        torch.cuda.empty_cache()
        line["breakdown"].update(other_legs(args, lib, dev, stream))
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def other_legs(args, lib, dev, stream):
    """The other configurations of the metric, each after the main timed
    region (its own clocks and timing; nothing here enters `value`):
      c1: n = 1001 latencies of PFTRF / PFTRS / PFTRI;
      mixed: n = 32768, nrhs = 64, kappa = 1e6, split-BF16 and split-TF32
             mixed-precision solves against FP64 PFTRF + PFTRS on the same
             matrix;
      batched: 4096 uneven matrices (n ~ U{32..512}), FP64 and FP32;
      serve: the request stream, saturation then Poisson arrivals at 0.7 of
             the measured capacity (2000 requests, at most 45 s of arrivals).
    A leg that fails records its error instead of its numbers."""
    import torch
    out = {}
    for leg in [x for x in args.legs.split(",") if x]:
        t0 = time.time()
        try:
            if leg == "c1":
                out["c1"] = c1_leg(lib, dev, stream)
            elif leg == "mixed":
                sampler = ClockSampler(0)
                sampler.start()
                fp64, res = mixed_leg(lib, dev, stream, 32768, 64, [1e6], ["bf16x6", "tf32x3"],
                                      30, True)
                out["mixed"] = {"workload": "n=32768, nrhs=64, kappa=1e6, A = Q diag(lam) Q^T "
                                            "(random butterfly Q, lam log-uniform on [1, 1e6])",
                                "fp64": fp64, "results": res, "clocks": sampler.stop()}
            elif leg == "batched":
                legs, arf_len, flops = batched_leg(lib, dev, 4096, ("f64", "f32"), 3, 10)
                out["batched"] = {"workload": "4096 SPD matrices, n ~ U{32..512}, 8 layouts, "
                                              "nrhs ~ U{1..8}; one graph-captured launch",
                                  "flops_per_batch": flops, **legs}
            elif leg == "serve":
                out["serve"] = serve_leg(lib, dev, 1000, 2000, 64, [0.7], resident_requests=500,
                                         load_time_cap_s=45.0)
            else:
                out[leg] = {"error": "unknown leg"}
        except Exception as exc:    # keep the main line; say what failed
            out[leg] = {"error": f"{type(exc).__name__}: {exc}"}
        out.setdefault(leg, {})["leg_wall_s"] = time.time() - t0
        torch.cuda.empty_cache()
    return out


def e2e_leg(args, lib, A, B0, dev, stream):
    """The same metric through the C ABI with host buffers: per step the RFP
    array and B go host -> device from pinned memory, PFTRF + PFTRS run, and
    X comes back device -> host."""
    import torch

    from paper_0901_1696_gb300.flops import pftrf_flops, pftrs_flops
    n, nrhs = args.n, args.nrhs
    nt = n * (n + 1) // 2
    arf_d = torch.empty(nt, dtype=torch.float64, device=dev)
    lib.rfp_dpack("N", "L", n, A, n, arf_d, stream)
    arf_h = torch.empty(nt, dtype=torch.float64, pin_memory=True)
    arf_h.copy_(arf_d)
    B_h = torch.empty_like(B0, device="cpu").pin_memory()
    B_h.copy_(B0)
    X_h = torch.empty_like(B_h).pin_memory()
    X_d = torch.empty_like(B0)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.e2e_steps):
        arf_d.copy_(arf_h, non_blocking=True)
        X_d.copy_(B_h, non_blocking=True)
        lib.rfp_dpftrf("N", "L", n, arf_d, info, stream)
        lib.rfp_dpftrs("N", "L", n, nrhs, arf_d, X_d, n, stream)
        X_h.copy_(X_d, non_blocking=True)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1) / args.e2e_steps
    assert int(info.item()) == 0
    return {"value": (pftrf_flops(n) + pftrs_flops(n, nrhs)) / (ms * 1e-3) / 1e12,
            "unit": "TFLOP/s", "h2d_bytes_per_step": nt * 8 + n * nrhs * 8,
            "d2h_bytes_per_step": n * nrhs * 8, "ms_per_step": ms}


def c1_leg(lib, dev, stream, reps: int = 30, oracle_too: bool = True):
    """The small latency-bound configuration: n = 1001 (odd), TRANSR = 'N',
    UPLO = 'L', A = B B^T / n + I (B ~ U[-1, 1], seed 0), PFTRF, PFTRS with
    nrhs = 16, PFTRI.  Each call is timed alone with CUDA events on the
    launching stream (median of `reps`, after 5 warm-up rounds); the 4 MB
    RFP array would stay in L2, so a 256 MB buffer is written (untimed)
    before every timed call.  The same three calls of the plain oracle on
    the host are timed once beside them."""
    import numpy as np
    import torch

    import rfp_inputs as gen
    n, nrhs = 1001, 16
    A, rng = gen.spd_bbt(n, seed=0, return_rng=True)
    Bh = gen.rhs(n, nrhs, rng)
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev)
    arf0 = torch.empty(n * (n + 1) // 2, dtype=torch.float64, device=dev)
    lib.rfp_dpack("N", "L", n, dA, n, arf0, stream)
    arf = torch.empty_like(arf0)
    fac = torch.empty_like(arf0)
    B0 = torch.from_numpy(np.ascontiguousarray(Bh.T)).to(dev)
    X = torch.empty_like(B0)
    info = torch.zeros(2, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    times = {"pftrf": [], "pftrs": [], "pftri": []}

    def timed(key, fn, record):
        flush.fill_(1)
        ev[0].record(stream)
        fn()
        ev[1].record(stream)
        if record:
            torch.cuda.synchronize(dev)
            times[key].append(ev[0].elapsed_time(ev[1]) * 1e3)

    for r in range(5 + reps):
        rec = r >= 5
        arf.copy_(arf0)
        timed("pftrf", lambda: lib.rfp_dpftrf("N", "L", n, arf, info[0:1], stream), rec)
        if r == 0:
            fac.copy_(arf)
        X.copy_(B0)
        timed("pftrs", lambda: lib.rfp_dpftrs("N", "L", n, nrhs, arf, X, n, stream), rec)
        timed("pftri", lambda: lib.rfp_dpftri("N", "L", n, arf, info[1:2], stream), rec)
    torch.cuda.synchronize(dev)
    assert int(info.abs().sum().item()) == 0
    Xh = X.cpu().numpy().T
    # per-step split (events between the steps; three extra rounds, not in
    # the medians above)
    lib.rfp_stage_timing(True)
    for _ in range(3):
        arf.copy_(arf0)
        flush.fill_(1)
        lib.rfp_dpftrf("N", "L", n, arf, info[0:1], stream)
        X.copy_(B0)
        lib.rfp_dpftrs("N", "L", n, nrhs, arf, X, n, stream)
        lib.rfp_dpftri("N", "L", n, arf, info[1:2], stream)
    torch.cuda.synchronize(dev)
    steps = {}
    for name, ms in lib.rfp_stage_times():
        steps[name] = steps.get(name, 0.0) + ms * 1e3 / 3
    lib.rfp_stage_timing(False)
    from paper_0901_1696_gb300.flops import pftrf_flops, pftri_flops, pftrs_flops
    med = {k: float(np.median(v)) for k, v in times.items()}
    out = {"workload": "n=1001 N/L, A = B B^T/n + I (seed 0), nrhs=16; L2 flushed before each call",
           **{f"{k}_us": v for k, v in med.items()},
           **{f"{k}_us_min": float(np.min(v)) for k, v in times.items()},
           "pftrf_gflops": pftrf_flops(n) / (med["pftrf"] * 1e-6) / 1e9,
           "pftrs_gflops": pftrs_flops(n, nrhs) / (med["pftrs"] * 1e-6) / 1e9,
           "pftri_gflops": pftri_flops(n) / (med["pftri"] * 1e-6) / 1e9,
           "bwd_err": sampled_backward_error(A, Xh, Bh), "reps": reps,
           "steps_us": {k: round(v, 1) for k, v in steps.items()}}
    if oracle_too:
        import oracle
        packed = oracle.pack("N", "L", A)
        t0 = time.perf_counter()
        ofac, oinfo = oracle.pftrf("N", "L", n, packed)
        t1 = time.perf_counter()
        oracle.pftrs("N", "L", n, ofac, Bh)
        t2 = time.perf_counter()
        oracle.pftri("N", "L", n, ofac)
        t3 = time.perf_counter()
        out["oracle_us"] = {"pftrf": (t1 - t0) * 1e6, "pftrs": (t2 - t1) * 1e6,
                            "pftri": (t3 - t2) * 1e6}
        out["max_abs_diff_factor_vs_oracle"] = float(np.max(np.abs(fac.cpu().numpy() - ofac)))
    return out


def sampled_backward_error(A, X, B):
    """max_j ||b_j - A x_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf) with a
    plain host FP64 residual (numpy) on the given columns."""
    import numpy as np
    R = B - A @ X
    anorm = float(np.max(np.sum(np.abs(A), axis=1)))
    den = anorm * np.max(np.abs(X), axis=0) + np.max(np.abs(B), axis=0)
    return float(np.max(np.max(np.abs(R), axis=0) / den))


def run_mixed(args):
    """Mixed-precision solve (low-precision factor + FP64 refinement) of an
    n = 32768 FP64 RFPF system with nrhs = 64, for each condition number and
    precision, against FP64 PFTRF + PFTRS on the same GPU (its own line)."""
    import torch

    from paper_0901_1696_gb300 import binding as rfp
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    lib = rfp.library()
    n, nrhs = args.mixed_n, args.mixed_nrhs
    fp64, results = mixed_leg(lib, dev, torch.cuda.current_stream(dev), n, nrhs,
                              [float(k) for k in args.kappas.split(",")], args.precs.split(","),
                              args.max_iter, not args.no_fp64_ref)
    line = {"mode": "mixed", "metric": "mixed-precision RFPF solve: time and backward error "
                                        "vs FP64 PFTRF+PFTRS",
            "unit": "ms", "higher_is_better": False, "n": n, "nrhs": nrhs, "dtype": "f64 in/out",
            "data": "synthetic: A = Q diag(lam) Q^T, Q random butterfly (n power of two) else "
                    "Haar, lam log-uniform on [1, kappa] with endpoints pinned",
            "tol": 1e-15, "fp64": fp64, "results": results}
    print(json.dumps(line), flush=True)


def mixed_leg(lib, dev, stream, n, nrhs, kappas, precs_wanted, max_iter, fp64_ref=True):
    """For each condition number: FP64 PFTRF + PFTRS (unless fp64_ref is
    False) and the mixed-precision solve in each precision, on the same
    matrix.  Errors: the device's backward error, a host FP64 residual on 4
    sampled columns, and the max-norm distance to the FP64 solution.
    Returns (fp64 rows, mixed rows)."""
    import numpy as np
    import torch

    import rfp_inputs as gen
    from paper_0901_1696_gb300 import binding as rfp
    from paper_0901_1696_gb300.flops import pftrf_flops, pftrs_flops
    precs = {"fp32": rfp.RFP_PREC_FP32, "tf32": rfp.RFP_PREC_TF32, "bf16": rfp.RFP_PREC_BF16,
             "tf32x3": rfp.RFP_PREC_TF32X3, "bf16x6": rfp.RFP_PREC_BF16X6}
    results, fp64 = [], []
    Bh = gen.rhs(n, nrhs, seed=3)
    dB = torch.from_numpy(np.ascontiguousarray(Bh.T)).to(dev)
    X = torch.empty_like(dB)
    status = torch.zeros(24, dtype=torch.uint8, device=dev)
    sample = [0, nrhs // 3, 2 * nrhs // 3, nrhs - 1]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for kappa in kappas:
        A = gen.spd_butterfly(n, seed=0, kappa=kappa, device=dev) if n & (n - 1) == 0 else \
            gen.spd_spectrum(n, seed=0, kappa=kappa, device=dev)
        arf = torch.empty(n * (n + 1) // 2, dtype=torch.float64, device=dev)
        lib.rfp_dpack("N", "L", n, A, n, arf, stream)
        Ah = A.cpu().numpy()
        del A
        X64h = None
        if not fp64_ref:
            fp64.append({"kappa": kappa, "skipped": True})
        # FP64 reference path on a copy
        fac = arf.clone() if fp64_ref else None
        ms64 = None
        if fac is not None:
            X64 = dB.clone()
            info = torch.zeros(1, dtype=torch.int32, device=dev)
            torch.cuda.synchronize(dev)
            ev[0].record(stream)
            lib.rfp_dpftrf("N", "L", n, fac, info, stream)
            lib.rfp_dpftrs("N", "L", n, nrhs, fac, X64, n, stream)
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            ms64 = ev[0].elapsed_time(ev[1])
            X64h = X64.cpu().numpy().T
            fp64.append({"kappa": kappa, "ms": ms64, "info": int(info.item()),
                         "tflops": (pftrf_flops(n) + pftrs_flops(n, nrhs)) / (ms64 * 1e-3) / 1e12,
                         "bwd_sampled": sampled_backward_error(Ah, X64h[:, sample], Bh[:, sample])})
            del fac, X64
        for name in precs_wanted:
            prec = precs[name]
            wb = lib.rfp_dpfsv_mixed_workspace(n, nrhs, prec)
            work = torch.empty(wb, dtype=torch.uint8, device=dev)
            for rep in range(2):            # first call warms up, second is timed
                torch.cuda.synchronize(dev)
                lib.rfp_stage_timing(True)
                ev[0].record(stream)
                lib.rfp_dpfsv_mixed("N", "L", n, nrhs, arf, dB, n, X, n, prec, max_iter,
                                    1e-15, work, wb, status, stream)
                ev[1].record(stream)
                torch.cuda.synchronize(dev)
                stages = {}
                for stage, t in lib.rfp_stage_times():
                    stages[stage] = stages.get(stage, 0.0) + t
                lib.rfp_stage_timing(False)
            ms = ev[0].elapsed_time(ev[1])
            st = rfp.mixed_status(status.cpu().numpy().tobytes())
            Xh = X.cpu().numpy().T
            fwd = float(np.max(np.abs(Xh - X64h)) / np.max(np.abs(X64h))) if X64h is not None else None
            results.append({
                "kappa": kappa, "prec": name, "ms": ms,
                "speedup_vs_fp64": ms64 / ms if ms64 else None,
                "steps_ms": {k.split(".")[1]: v for k, v in stages.items()},
                "iterations": st["iterations"], "converged": st["converged"],
                "info": st["info"], "tc_error": st["tc_error"],
                "backward_error": st["backward_error"],
                "bwd_sampled": sampled_backward_error(Ah, Xh[:, sample], Bh[:, sample])
                if st["info"] == 0 else None,
                "fwd_vs_fp64": fwd,
                "factor_tflops": pftrf_flops(n) / (stages.get("mixed.factor", 0) * 1e-3) / 1e12
                if stages.get("mixed.factor") else None})
            del work
        del arf, Ah
        torch.cuda.empty_cache()
    return fp64, results


def run_batched(args):
    """Batched PFTRF + PFTRS: `--batch` independent SPD matrices of uneven
    order n ~ U{32..512}, each in one of the 8 layouts (uniform), nrhs ~
    U{1..8}, A_k = B B^T / n + I (rfp_inputs.spd_bbt, seed 1000 + k), in
    FP64 and in FP32, one graph-captured launch per batch.  The panel width
    per n-bucket comes from the autotuner's cache, else from the table
    shipped for the GPU model, else it is tuned on first use."""
    import torch

    from paper_0901_1696_gb300 import binding as rfp

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    lib = rfp.library()
    count = args.batch
    legs, arf_len, flops = batched_leg(lib, dev, count, ("f64", "f32"), args.warmup, args.steps,
                                       args.retune)
    line = {"mode": "batched", "metric": "batched PFTRF+PFTRS TFLOP/s (uneven SPD RFPF batch)",
            "value": legs["f64"]["tflops"], "unit": "TFLOP/s", "higher_is_better": True,
            "steps": args.steps, "warmup": args.warmup, "dtype": "f64",
            "data": "synthetic: A_k = B B^T / n + I, B ~ U[-1,1] (numpy PCG64, seed 1000 + k)",
            "config": {"workload": f"{count} SPD matrices, n ~ U{{32..512}}, 8 layouts uniform, "
                                   "nrhs ~ U{1..8}; one graph-captured launch per batch",
                       "batch": count, "flops_per_batch": flops,
                       "l2": "inputs restored before every replay (untimed copy of "
                             f"{arf_len * 8 / 1e9:.2f} GB FP64 > L2)"},
            **legs}
    print(json.dumps(line), flush=True)


def batched_leg(lib, dev, count, precs, warmup, steps, retune=False):
    """Batched PFTRF + PFTRS of `count` uneven matrices in each precision of
    `precs` ("f64", "f32"); returns ({prec: leg}, arf_len, flops)."""
    import numpy as np
    import torch

    import rfp_inputs as gen
    from paper_0901_1696_gb300 import batched as bt
    from paper_0901_1696_gb300.flops import pftrf_flops, pftrs_flops
    from paper_0901_1696_gb300.peaks import FP32_FMA_PER_SM_CLK, SM_COUNT, SM_MAX_MHZ

    gpu = torch.cuda.get_device_properties(dev).name
    rng = np.random.default_rng(0)
    ns = [int(x) for x in rng.integers(32, 513, count)]
    lay = rng.integers(0, 8, count)
    layouts = [("N", "L"), ("N", "U"), ("T", "L"), ("T", "U")]
    transrs = [layouts[int(x) % 4][0] for x in lay]
    uplos = [layouts[int(x) % 4][1] for x in lay]
    nrhss = [int(x) for x in rng.integers(1, 9, count)]
    # (the 8 layouts: 4 TRANSR x UPLO pairs x the parity of n, which n's own draw sets)
    entries, arf_len, b_len = bt.make_entries(ns, transrs, uplos, nrhss)
    flops = sum(pftrf_flops(n) + pftrs_flops(n, r) for n, r in zip(ns, nrhss))
    sample = sorted(set(int(x) for x in np.linspace(0, count - 1, 12)))
    kept = {}
    legs = {}
    for prec, dtype in (("f64", torch.float64), ("f32", torch.float32)):
        if prec not in precs:
            continue
        arf = torch.empty(max(arf_len, 1), dtype=dtype, device=dev)
        B = torch.empty(max(b_len, 1), dtype=dtype, device=dev)
        pack = lib.rfp_dpack if dtype == torch.float64 else lib.rfp_spack
        t_gen = time.time()
        for k in range(count):
            n, r = ns[k], nrhss[k]
            A, r2 = gen.spd_bbt(n, seed=1000 + k, return_rng=True)
            Bk = gen.rhs(n, r, r2)
            if k in sample:
                kept[k] = (A, Bk)
            dA = torch.from_numpy(A).to(dev, dtype)
            pack(transrs[k], uplos[k], n, dA, n, arf[int(entries["arf"][k]):])
            off = int(entries["b"][k])
            B[off: off + n * r] = torch.from_numpy(Bk.ravel(order="F")).to(dev, dtype)
        torch.cuda.synchronize(dev)
        t_gen = time.time() - t_gen
        cache = bt.TuningCache()
        tuned = False
        if retune or not cache.get(gpu, prec):
            bt.autotune(prec, cache=cache)
            tuned = True
        cache.fill_nb(entries, gpu, prec)
        # warm-up replays, then timed replays; inputs restored before each (not timed)
        sampler = ClockSampler(0)
        t0 = time.time()
        bt.time_batch(torch, lib, entries, arf, B, dtype, reps=max(warmup, 1))
        sampler.start()
        ms, out_a, out_b, info = bt.time_batch(torch, lib, entries, arf, B, dtype,
                                               reps=max(steps, 1))
        clocks = sampler.stop()
        wall = time.time() - t0
        info_h = info.cpu().numpy()
        bh = out_b.cpu().numpy().astype(np.float64)
        bwd = 0.0
        for k in sample:
            A, Bk = kept[k]
            n, r = ns[k], nrhss[k]
            off = int(entries["b"][k])
            Xk = bh[off: off + n * r].reshape(r, n).T
            bwd = max(bwd, sampled_backward_error(A, Xk, Bk))
        mhz = clocks["sm_mhz"] or SM_MAX_MHZ
        if prec == "f64":
            peak, bound = fp64_peak_tflops(mhz), "FP64 FMA pipe: 152 SMs x 2 FMA x 2 x clock"
        else:
            peak = SM_COUNT * FP32_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12
            bound = "FP32 FMA pipe: 152 SMs x 128 FMA x 2 x clock"
        tflops = flops / (ms * 1e-3) / 1e12
        legs[prec] = {
            "ms": ms, "tflops": tflops, "matrices_per_s": count / (ms * 1e-3),
            "roofline": {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "traffic": None, "kernel": "batched_kernel",
                         "peak_source": bound},
            "info_nonzero": int(np.count_nonzero(info_h)), "bwd_sampled_max": bwd,
            "nb_table": cache.get(gpu, prec), "nb_table_source": cache.source(gpu, prec),
            "autotuned_now": tuned, "clocks": clocks, "gen_s": t_gen, "wall_s": wall}
        del arf, B, out_a, out_b
        torch.cuda.empty_cache()
    return legs, arf_len, flops


def run_serve(args):
    """Serving loop (rfp_serve_*) on its own line: closed-loop saturation to
    measure capacity, Poisson arrivals at the given fractions of it, then
    solve requests on resident factors (serve_leg)."""
    import torch

    from paper_0901_1696_gb300 import binding as rfp
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    lib = rfp.library()
    R, P = args.serve_requests, args.serve_pool
    loads = [float(x) for x in args.serve_loads.split(",") if x]
    out = serve_leg(lib, dev, R, R, P, loads, resident_requests=min(R, 1000))
    line = {"mode": "serve", "metric": "served solves/s, p50/p99 at <=1e-12 bwd err",
            "value": out["runs"]["saturation"]["solves_per_s"], "unit": "solves/s (right-hand sides)",
            "higher_is_better": True, "dtype": "f64 in/out (FP64 or split-BF16 + FP64 refinement)",
            "data": "synthetic: A = Q diag(lam) Q^T, Q = 8 Householder reflectors, lam log-uniform "
                    "on [1, kappa]",
            "config": {"workload": out["workload"], "requests": R, "pool": P},
            **{k: v for k, v in out.items() if k != "workload"}}
    print(json.dumps(line), flush=True)


def serve_leg(lib, dev, sat_requests, load_requests, pool_size, loads, resident_requests=0,
              load_time_cap_s=None):
    """A stream of factor+solve requests through the serving loop: n
    log-uniform in [64, 8192], kappa log-uniform in [1e1, 1e6], nrhs ~
    U{1..32}, layouts uniform, FP64 / mixed-precision modes uniform, host
    inputs in pinned memory, drawn from a pool of `pool_size` matrices.
    Runs: closed-loop saturation (`sat_requests` submitted at t = 0) to
    measure capacity, then Poisson arrivals at each fraction in `loads` of it
    (`load_requests` each, fewer if the arrivals would last longer than
    `load_time_cap_s`), then `resident_requests` solves on resident factors.
    Latency = done - submit on the server's host clock.  Backward errors of
    48 sampled requests of the saturation run are checked by a plain FP64
    residual on the device against the unpacked matrix."""
    import numpy as np
    import torch

    import rfp_inputs as gen
    from paper_0901_1696_gb300 import batched as bt
    from paper_0901_1696_gb300 import serve as sv

    R = max(sat_requests, load_requests, resident_requests)
    P = pool_size
    rng = np.random.default_rng(0)
    layouts = [("N", "L"), ("N", "U"), ("T", "L"), ("T", "U")]
    pool = []
    for i in range(P):
        n = int(round(np.exp(rng.uniform(np.log(64), np.log(8192)))))
        kappa = float(10 ** rng.uniform(1, 6))
        t, u = layouts[int(rng.integers(0, 4))]
        A = gen.spd_reflectors(n, seed=500 + i, kappa=kappa, device=dev)
        arf_d = torch.empty(n * (n + 1) // 2, dtype=torch.float64, device=dev)
        lib.rfp_dpack(t, u, n, A, n, arf_d)
        del A
        pool.append(dict(n=n, kappa=kappa, t=t, u=u, arf_d=arf_d,
                         arf_h=arf_d.cpu().pin_memory()))
    torch.cuda.synchronize(dev)
    which = rng.integers(0, P, R)
    nrhs = rng.integers(1, 33, R)
    modes = rng.integers(0, 2, R)
    sizes = [pool[int(w)]["n"] * int(r) for w, r in zip(which, nrhs)]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    Bh = torch.from_numpy(rng.uniform(-1, 1, int(offs[-1]))).pin_memory()
    Xh = torch.zeros(int(offs[-1]), dtype=torch.float64).pin_memory()
    gpu = torch.cuda.get_device_properties(dev).name
    table = bt.TuningCache().get(gpu, "f64")
    nb = [[(table or {}).get(t, [16] * 8)[b] for b in range(8)] for t in ("N", "T")]
    arena = 150 << 30

    def one_run(count, arrivals, key_base):
        """The first `count` requests; arrivals: submit times (s) relative to
        the start, or None (all at once)."""
        Xh.zero_()
        with sv.Server(arena_bytes=arena, streams=8, batch_max=1024, small_n=512,
                       max_iter=30, tol=1e-15, batch_nb=nb) as s:
            t0 = time.perf_counter()
            for k in range(count):
                if arrivals is not None:
                    dt = arrivals[k] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                pm = pool[int(which[k])]
                n, r = pm["n"], int(nrhs[k])
                s.submit(k, sv.OP_FACTOR_SOLVE, int(modes[k]), pm["t"], pm["u"], n, r,
                         arf=pm["arf_h"].data_ptr(),
                         B=Bh.data_ptr() + 8 * int(offs[k]), X=Xh.data_ptr() + 8 * int(offs[k]),
                         key=key_base + k)
            done = s.wait(count, timeout=1800)
            st = s.stats()
        done.sort(key=lambda c: c["id"])
        lat = np.array([c["t_done"] - c["t_submit"] for c in done]) * 1e3
        span = max(c["t_done"] for c in done) - min(c["t_submit"] for c in done)
        ok = [c["status"] == 0 for c in done]
        fp64 = modes[:count] == 0
        # device concurrency from the per-request device stamps: the mean
        # number of requests in progress on the GPU over the span of GPU work
        iv = sorted((c["gpu_start_ms"], c["gpu_end_ms"]) for c in done if c["gpu_end_ms"] > 0)
        gspan = (max(e for _, e in iv) - iv[0][0]) if iv else 0.0
        conc = sum(e - b for b, e in iv) / gspan if gspan > 0 else 0.0
        return {"requests": count, "requests_per_s": count / span,
                "mean_requests_in_progress_on_gpu": conc,
                "solves_per_s": float(nrhs[:count].sum()) / span,
                "span_s": span, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "p50_fp64_ms": float(np.percentile(lat[fp64], 50)),
                "p99_fp64_ms": float(np.percentile(lat[fp64], 99)),
                "p50_mixed_ms": float(np.percentile(lat[~fp64], 50)),
                "p99_mixed_ms": float(np.percentile(lat[~fp64], 99)),
                "ok": int(sum(ok)), "failed": int(count - sum(ok)),
                "statuses": sorted(set(int(c["status"]) for c in done)),
                "batched_fraction": st["batched_requests"] / count,
                "mean_batch": st["batched_requests"] / max(st["batches"], 1),
                "evictions": st["evictions"], "cache_gb": st["cache_bytes"] / 1e9}, done

    runs = {}
    sampler = ClockSampler(0)
    sampler.start()
    sat, done = one_run(sat_requests, None, 0)
    runs["saturation"] = sat
    # sampled backward errors of the saturation run: FP64 residual on the GPU
    check = sorted(set(int(x) for x in np.linspace(0, sat_requests - 1, 48)))
    bwd = []
    for k in check:
        pm = pool[int(which[k])]
        n, r = pm["n"], int(nrhs[k])
        Af = torch.zeros(n, n, dtype=torch.float64, device=dev)
        lib.rfp_dunpack(pm["t"], pm["u"], n, pm["arf_d"], Af, n)   # one triangle (row-major view)
        Af = Af + Af.T - torch.diag(torch.diagonal(Af))
        B = Bh[int(offs[k]): int(offs[k]) + n * r].to(dev).view(r, n).T
        X = Xh[int(offs[k]): int(offs[k]) + n * r].to(dev).view(r, n).T
        res = (B - Af @ X).abs().amax(0)
        den = Af.abs().sum(1).amax() * X.abs().amax(0) + B.abs().amax(0)
        bwd.append(dict(k=k, n=n, mode=int(modes[k]), bwd=float((res / den).max())))
        del Af
    cap = sat["requests_per_s"]
    for f in loads:
        count = load_requests
        if load_time_cap_s:
            count = max(1, min(count, int(f * cap * load_time_cap_s)))
        gaps = np.random.default_rng(7).exponential(1.0 / (f * cap), count)
        runs[f"load_{f:g}"] = one_run(count, np.cumsum(gaps) - gaps[0],
                                      10 ** 7 * (1 + len(runs)))[0]
        runs[f"load_{f:g}"]["offered_requests_per_s"] = f * cap
    if resident_requests:
        # solve requests on resident factors (cache hits): FP64 factors of the pool
        with sv.Server(arena_bytes=arena, streams=8, batch_max=1024, small_n=512,
                       batch_nb=nb) as s:
            prime_x = torch.zeros(sum(pm["n"] for pm in pool), dtype=torch.float64).pin_memory()
            po = np.concatenate([[0], np.cumsum([pm["n"] for pm in pool])])
            for i, pm in enumerate(pool):
                s.submit(i, sv.OP_FACTOR_SOLVE, sv.MODE_FP64, pm["t"], pm["u"], pm["n"], 1,
                         arf=pm["arf_h"].data_ptr(), B=Bh.data_ptr(),
                         X=prime_x.data_ptr() + 8 * int(po[i]), key=i)
            s.wait(P)
            m = resident_requests
            for k in range(m):
                i = int(which[k])
                pm = pool[i]
                s.submit(P + k, sv.OP_SOLVE, sv.MODE_FP64, pm["t"], pm["u"], pm["n"],
                         int(nrhs[k]), B=Bh.data_ptr() + 8 * int(offs[k]),
                         X=Xh.data_ptr() + 8 * int(offs[k]), key=i)
            hits = s.wait(m)
        hl = np.array([c["t_done"] - c["t_submit"] for c in hits]) * 1e3
        hspan = max(c["t_done"] for c in hits) - min(c["t_submit"] for c in hits)
        runs["resident_solves"] = {
            "requests": m, "submitted": "all at once (latency includes queueing)",
            "solves_per_s": float(nrhs[:m].sum()) / hspan, "requests_per_s": m / hspan,
            "cache_hit_fraction": float(np.mean([c["cache_hit"] for c in hits])),
            "p50_ms": float(np.percentile(hl, 50)), "p99_ms": float(np.percentile(hl, 99)),
            "ok": int(sum(c["status"] == 0 for c in hits))}
    clocks = sampler.stop()
    worst = max(b["bwd"] for b in bwd)
    return {"workload": f"factor+solve requests over {P} matrices, n log-uniform [64, 8192], "
                        "kappa log-uniform [1e1, 1e6], nrhs ~ U{1..32}, layouts uniform, FP64 / "
                        "mixed uniform; arena 150 GB, 8 streams + batched launches for small "
                        "FP64 requests",
            "runs": runs,
            "bwd_sampled": {"count": len(bwd), "max": worst, "all_le_1e-12": bool(worst <= 1e-12),
                            "max_mixed": max([b["bwd"] for b in bwd if b["mode"] == 1] or [0.0])},
            "clocks": clocks}


def run_surface(args):
    """The rest of the LAPACK 3.2 RFP surface at the bench's order (FP64, one
    layout pair per routine): TPTTF / TFTTP and LANSF against HBM bandwidth
    (their algorithmic bytes: read + write of the packed and RFP arrays; one
    read of the RFP array per row pass of LANSF's two), SFRK and TFSM against
    the FP64 pipe (n^2 k and m^2 nc flops times 2 / 1), TFTRI by time (n^3/3
    flops).  Event-timed, median of `--steps` after `--warmup`."""
    import numpy as np
    import torch

    import rfp_inputs as gen
    from paper_0901_1696_gb300 import binding as rfp

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    lib = rfp.library()
    n = args.n
    nt = n * (n + 1) // 2
    peaks = {}
    mp = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    if os.path.exists(mp):
        with open(mp) as f:
            peaks = json.load(f)
    hbm = peaks.get("hbm_gbs", 6800.0)
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    ap = torch.rand(nt, dtype=torch.float64, device=dev, generator=g)
    arf = torch.empty(nt, dtype=torch.float64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, reps=None):
        reps = reps or max(args.steps, 3)
        for _ in range(max(args.warmup, 1)):
            fn()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            ev[0].record()
            fn()
            ev[1].record()
            torch.cuda.synchronize(dev)
            ts.append(ev[0].elapsed_time(ev[1]))
        return float(np.median(ts))

    sampler = ClockSampler(0)
    sampler.start()
    out = {}
    ms = timed(lambda: lib.rfp_dtpttf("N", "L", n, ap, arf))
    out["tpttf"] = {"ms": ms, "gbs": 16 * nt / (ms * 1e-3) / 1e9}
    back = torch.empty_like(ap)
    ms = timed(lambda: lib.rfp_dtfttp("T", "U", n, arf, back))
    out["tfttp"] = {"ms": ms, "gbs": 16 * nt / (ms * 1e-3) / 1e9}
    work = torch.empty(2 * n, dtype=torch.float64, device=dev)
    val = torch.empty(1, dtype=torch.float64, device=dev)
    for norm in ("M", "1", "F"):
        ms = timed(lambda: lib.rfp_dlansf(norm, "N", "L", n, arf, work, val))
        reads = 8 * nt * (2 if norm != "F" else 4)   # each row reads its full symmetric row once (twice for F)
        out[f"lansf_{norm}"] = {"ms": ms, "gbs_algorithmic": 8 * nt / (ms * 1e-3) / 1e9,
                                "gbs_touched": reads / (ms * 1e-3) / 1e9}
    k = 256
    A = torch.rand(n, k, dtype=torch.float64, device=dev, generator=g)   # row-major n x k = col-major k x n
    ms = timed(lambda: lib.rfp_dsfrk("N", "L", "T", n, k, 1.0, A, k, 1.0, arf))
    out["sfrk"] = {"ms": ms, "k": k, "tflops": float(n) * (n + 1) * k / (ms * 1e-3) / 1e12}
    # TFSM with a well-conditioned triangle: the factor of the bench's matrix
    Afull = gen.spd_butterfly(n, seed=0, kappa=1e4, device=dev) if n & (n - 1) == 0 else \
        gen.spd_spectrum(n, seed=0, kappa=1e4, device=dev)
    lib.rfp_dpack("N", "L", n, Afull, n, arf)
    del Afull
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    lib.rfp_dpftrf("N", "L", n, arf, info)
    nc = 256
    B0 = torch.rand(nc, n, dtype=torch.float64, device=dev, generator=g)
    B = B0.clone()
    ms = timed(lambda: (B.copy_(B0), lib.rfp_dtfsm("N", "L", "L", "N", "N", n, nc, 1.0, arf, B, n)))
    ms_copy = timed(lambda: B.copy_(B0))
    out["tfsm"] = {"ms": ms - ms_copy, "nrhs": nc,
                   "tflops": float(n) * n * nc / ((ms - ms_copy) * 1e-3) / 1e12}
    fac = arf.clone()
    ms = timed(lambda: (arf.copy_(fac), lib.rfp_dtftri("N", "L", "N", n, arf, info)), reps=3)
    ms_copy = timed(lambda: arf.copy_(fac))
    out["tftri"] = {"ms": ms - ms_copy, "tflops": n ** 3 / 3 / ((ms - ms_copy) * 1e-3) / 1e12}
    clocks = sampler.stop()
    fp64 = fp64_peak_tflops(clocks["sm_mhz"])
    for key in ("tpttf", "tfttp"):
        out[key]["frac_of_hbm"] = out[key]["gbs"] / hbm
    for key in ("sfrk", "tfsm", "tftri"):
        out[key]["frac_of_fp64_pipe"] = out[key]["tflops"] / fp64
    line = {"mode": "surface", "metric": "LAPACK 3.2 RFP surface at n = %d (FP64)" % n,
            "unit": "mixed (see each routine)", "n": n, "hbm_peak_gbs": hbm,
            "fp64_peak_tflops": fp64, "routines": out, "clocks": clocks,
            "data": "synthetic: uniform [0, 1) arrays; TFSM / TFTRI on the factor of the bench matrix"}
    print(json.dumps(line), flush=True)


def run_c1(args):
    """The n = 1001 latency case alone (its own line): `--steps` timed calls
    of each routine after 5 warm-up rounds, without the oracle."""
    import torch

    from paper_0901_1696_gb300 import binding as rfp
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    out = c1_leg(rfp.library(), dev, torch.cuda.current_stream(dev), reps=max(args.steps, 1),
                 oracle_too=False)
    print(json.dumps({"mode": "c1", "metric": "PFTRF / PFTRS / PFTRI latency at n = 1001",
                      "unit": "us", "higher_is_better": False, **out}), flush=True)


def main():
    args = parse()
    if args.mode == "c1":
        run_c1(args)
        return
    if args.mode == "mixed":
        run_mixed(args)
        return
    if args.mode == "batched":
        run_batched(args)
        return
    if args.mode == "serve":
        run_serve(args)
        return
    if args.mode == "surface":
        run_surface(args)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if args.gpus == 1 else 1))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world)


if __name__ == "__main__":
    main()
