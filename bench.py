#!/usr/bin/env python
"""Benchmark of the EBC Greedy hot path on one GB300 (or N replicas).

Workload (default): drifting-regime sensor features, n = 200,000, d = 128,
Greedy k = 100, all points candidates.  One step = the instance prologue
(V device-to-device into the resident slot, norms, quantised copy, m_v) plus
k certified Greedy rounds.  Metric: distance evaluations per second, one
evaluation being one (candidate, point) pair of a round's bulk gains,
summed over rounds as sum_t (n - t) * n.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16|fp16|fp8|fp32]
    python bench.py --impl reference      # the CPU oracle on the same metric

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EBC distance-evals/s, BF16-TC vs FP32 plain at matched picks; serve p99 ms"
UNIT = "distance-evals/s"
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) per launch of the bulk kernel from one ncu capture
# of the current kernel at the full size (profiles/k_gains_tc_bf16_regime_d128.md),
# keyed by (precision, n, d); None where no capture of the current kernel exists.
NCU_TRAFFIC = {("bf16", 200_000, 128): 317.964032e6 + 11.459840e6}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            j = json.load(fh)
        return {"hbm_gbs": j["hbm_gbs"], "bf16": j["bf16_tflops"], "bf16_sustained": j["bf16_tflops_sustained"],
                "sm_max_mhz": j.get("sm_max_mhz", 2070.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def measure_fp8_peak(n: int = 8192, reps: int = 10, loop_s: float = 2.0):
    """Dense FP8 e4m3 tensor throughput of the library GEMM on this GPU, measured
    the way the BF16 peaks are: torch._scaled_mm (cuBLASLt) on n^3, best of
    `reps` timed with CUDA events (burst), and back to back for about loop_s
    seconds (sustained).  TFLOP/s; None where the library call is missing."""
    import torch
    try:
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()  # column-major operand
        one = torch.ones((), device="cuda")
        mm = lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        for _ in range(3):
            mm()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            mm()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        iters = max(1, int(loop_s * 1e3 / best))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(iters):
            mm()
        e1.record()
        torch.cuda.synchronize()
        flops = 2.0 * n ** 3
        return {"burst": flops / (best * 1e-3) / 1e12, "sustained": flops * iters / (e0.elapsed_time(e1) * 1e-3) / 1e12,
                "how": f"torch._scaled_mm e4m3 {n}^3 (2 n^3 flops): best of {reps} (burst) and {iters} back to back "
                       f"(sustained), CUDA events"}
    except Exception as ex:  # pragma: no cover - library without FP8 GEMM
        return {"burst": None, "sustained": None, "how": f"unavailable: {type(ex).__name__}"}


class ClockSampler:
    """nvidia-smi sampler run during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --- multi-rank helpers (one process per GPU; no collective on the data path) ---
def rank_env():
    """(world, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(seed: int, rank: int) -> int:
    """Each replica draws its own instance of the same shape."""
    return seed + rank


def shard(items, rank: int, world: int):
    """Whole instances are routed to ranks round-robin: disjoint, and together
    every instance exactly once."""
    return list(items)[rank::world]


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Timing of the slowest rank (the job ends when the last rank does)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def greedy_evals(n: int, k: int) -> int:
    return sum((n - t) * n for t in range(k))


def make_workload(args, rank: int):
    from paper_2105_12026_gb300 import synth
    if args.workload == "regime":
        w = synth.regime_greedy(seed=rank_seed(args.seed, rank), n=args.n, d=args.d, k=args.k)
        name = f"greedy drifting-regime features n={args.n} d={args.d} k={args.k}"
    else:
        w = synth.plain_greedy_small(seed=rank_seed(args.seed, rank), n=args.n, d=args.d)
        w["k"] = args.k
        name = f"greedy 8-cluster GMM n={args.n} d={args.d} k={args.k}"
    return w["V"], w["k"], name


def cpu_baseline(V, budget_s: float, seed: int = 0):
    """Oracle (FP64, all host threads) gains at S = {} on a sample of candidates."""
    import oracle
    n = V.shape[0]
    m = oracle.norms(V)
    rng = np.random.default_rng(seed)
    count, elapsed, done = 4, 0.0, 0
    t_all = time.perf_counter()
    while True:
        cand = rng.choice(n, size=count, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        oracle.gains(V, m, cand)
        dt = time.perf_counter() - t0
        elapsed += dt
        done += count
        if time.perf_counter() - t_all + 2.2 * dt > budget_s:
            break
        count = min(count * 2, n)
    return {"value": done * n / elapsed, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"oracle gains at S={{}} for {done} sampled candidates x all {n} points, FP64, "
                      f"{oracle.num_threads()} threads, {elapsed:.1f}s"}


def run_reference(args):
    """--impl reference: the CPU oracle on the same metric, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    V, k, name = make_workload(args, 0)
    n = V.shape[0]
    m = oracle.norms(V)
    rng = np.random.default_rng(1)
    per_step = max(1, int(args.ref_cands))
    times = []
    for s in range(args.warmup + args.steps):
        cand = rng.choice(n, size=per_step, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        oracle.gains(V, m, cand)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = args.steps * per_step * n / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": name, "sample": f"{per_step} candidates x {n} points per step (S = {{}})"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{per_step} sampled candidates x all {n} points per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def instance_evals(n: int, k: int) -> int:
    return greedy_evals(n, k)


def run_mix(args):
    """256 independent Greedy instances (n log-uniform 2k..100k, d in {16,32,64,128},
    k in 5..50).  --mix-mode group (default): resident handles, one step =
    re-upload every instance's V from pinned host memory (ebc_reload) and run
    every instance's rounds through ebc_group_greedy (one persistent bulk
    launch per round over all instances still running); streams: the same
    resident handles, each instance's rounds through ebc_greedy on its own
    stream (per-instance graphs); batch: the batch runtime (submit all, run to
    completion, handles created at admission)."""
    if args.mix_mode != "batch":
        return run_mix_resident(args)
    import torch
    import torch.distributed as dist

    from paper_2105_12026_gb300 import ebc, synth
    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    all_specs = synth.instance_mix(seed=args.seed, count=args.instances)
    specs = shard(all_specs, rank, world)  # whole instances per rank
    t0 = time.perf_counter()
    Vs = [sp.make() for sp in specs]
    gen_s = time.perf_counter() - t0
    evals = sum(instance_evals(sp.n, sp.k) for sp in all_specs)

    def one_batch():
        with ebc.Batch(max_slots=args.slots, budget_bytes=int(args.budget_gb * (1 << 30)),
                       refine_k=args.refine_k) as b:
            tickets = [b.submit(V, sp.k, args.prec) for V, sp in zip(Vs, specs)]
            b.run()
            for t in tickets:
                assert b.poll(t) is not None
            return b.stats()

    for _ in range(args.warmup):
        one_batch()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    for _ in range(args.steps):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        st = one_batch()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t1)
    clk = clocks.stop()
    tot = max_over_ranks(sum(times), world, dev)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": args.steps * evals / tot, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": args.prec, "data": "synthetic (seeded GMM instance mix)",
            "config": {"workload": f"batched greedy, {len(specs)} instances: n log-uniform [2000, 100000], "
                                   f"d in {{16,32,64,128}}, k in [5, 50]",
                       "slots": args.slots, "budget_gb": args.budget_gb, "evals_per_step": evals,
                       "parallelism": f"instances sharded over {world} GPUs" if world > 1 else "single GPU",
                       "timing": "wall clock between device synchronisations; includes host-to-device upload of "
                                 "every instance and the result copies",
                       "host_generation_s": gen_s},
            "batch_stats": st, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_mix_resident(args):
    import torch
    import torch.distributed as dist

    from paper_2105_12026_gb300 import ebc, synth
    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    all_specs = synth.instance_mix(seed=args.seed, count=args.instances)
    specs = shard(all_specs, rank, world)  # whole instances per rank
    t0 = time.perf_counter()
    Vs = [torch.from_numpy(sp.make()).pin_memory() for sp in specs]
    gen_s = time.perf_counter() - t0
    evals = sum(instance_evals(sp.n, sp.k) for sp in all_specs)
    ks = [sp.k for sp in specs]
    insts = [ebc.Instance(V, precision=args.prec, refine_k=args.refine_k, stream=torch.cuda.Stream())
             for V in Vs]
    outs = [(torch.empty(k, dtype=torch.int32, device=dev), torch.empty(k, dtype=torch.float64, device=dev))
            for k in ks]
    group = ebc.Group(lanes=args.group_lanes, by_row_width=args.group_by_width, max_ctas=args.group_ctas)

    def one_step():
        for inst, V in zip(insts, Vs):
            inst.reload(V)
        if args.mix_mode == "group":
            res = group.greedy(insts, ks)
        else:
            res = []
            for inst, k, (oi, of) in zip(insts, ks, outs):
                ebc.ebc_greedy(inst.h, k, oi.data_ptr(), of.data_ptr())
                res.append((oi, of))
        for inst in insts:
            inst.sync()
        return res

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    group.profiling(True)  # event pairs around the shared launches only
    group.reset_profile()
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    for _ in range(args.steps):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        res = one_step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t1)
    clk = clocks.stop()
    picks = [r[0].cpu().numpy().tolist() for r in res[:4]]
    gst = group.stats()
    gprof = group.profile()
    group.close()
    for inst in insts:
        inst.close()
    tot = max_over_ranks(sum(times), world, dev)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    h2d = sum(V.numel() * 4 for V in Vs)
    line = {"metric": METRIC, "value": args.steps * evals / tot, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": args.prec, "data": "synthetic (seeded GMM instance mix)",
            "config": {"workload": f"batched greedy, {len(specs)} instances: n log-uniform [2000, 100000], "
                                   f"d in {{16,32,64,128}}, k in [5, 50]",
                       "mix_mode": args.mix_mode, "group_lanes": args.group_lanes, "group_ctas": args.group_ctas,
                       "evals_per_step": evals,
                       "parallelism": f"instances sharded over {world} GPUs" if world > 1 else "single GPU",
                       "timing": "wall clock between device synchronisations; every step uploads each instance's "
                                 "V from pinned host memory into its resident handle (ebc_reload: prologue and "
                                 "quantisation included) and runs all its Greedy rounds",
                       "h2d_bytes_per_step": h2d, "host_generation_s": gen_s},
            "group_stats": gst if args.mix_mode == "group" else None,
            "shared_launches": ({"ms_per_step": gprof["launch_ms"] / args.steps,
                                 "gap_ms_per_step": gprof["gap_ms"] / args.steps,
                                 "pairs_per_s": gprof["pairs"] / (gprof["launch_ms"] * 1e-3)}
                                if args.mix_mode == "group" and gprof["launch_ms"] > 0 else None),
            "first_picks": picks, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Poisson arrivals through the batch runtime (continuous batching at round
    granularity); latency = completion - arrival, queueing included."""
    # many slot streams: let each have its own hardware queue (read at context creation)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch

    from paper_2105_12026_gb300 import ebc, synth
    torch.cuda.set_device(0)
    trace = synth.request_trace(seed=args.seed, rate=args.rate, horizon_s=args.horizon, large_frac=args.large_frac,
                                large_n=args.large_n)
    t0 = time.perf_counter()
    Vs = [r.spec.make() for r in trace]
    gen_s = time.perf_counter() - t0
    # warm the library (kernels, graphs) on a small instance
    with ebc.Batch(max_slots=2) as b:
        t = b.submit(Vs[0], min(3, trace[0].spec.k), args.prec)
        b.run()
        b.poll(t)
    b = ebc.Batch(max_slots=args.slots, budget_bytes=int(args.budget_gb * (1 << 30)), refine_k=args.refine_k)
    b.set_large(args.large_threshold, args.large_ctas, args.max_large)
    b.set_lazy(not args.no_lazy, args.lazy_min_n)
    pending = {}
    lat = {}
    nxt = 0
    clocks = ClockSampler(0)
    clocks.start()
    start = time.perf_counter()
    deadline = start + args.horizon + args.drain
    while True:
        now = time.perf_counter() - start
        while nxt < len(trace) and trace[nxt].t_arrive <= now:
            pending[b.submit(Vs[nxt], trace[nxt].spec.k, args.prec)] = nxt
            nxt += 1
        active, queued = b.step()
        for tk in list(pending):
            res = b.poll(tk)
            if res is not None:
                i = pending.pop(tk)
                lat[i] = (time.perf_counter() - start) - trace[i].t_arrive
        if nxt == len(trace) and not pending:
            break
        if time.perf_counter() > deadline:
            break
        if active == 0 and queued == 0 and nxt < len(trace):
            time.sleep(max(0.0, min(0.002, trace[nxt].t_arrive - (time.perf_counter() - start))))
    wall = time.perf_counter() - start
    clk = clocks.stop()
    st = b.stats()
    b.close()
    done = sorted(lat)
    lat_ms = np.array([1e3 * lat[i] for i in done]) if done else np.zeros(0)
    small = np.array([1e3 * lat[i] for i in done if not trace[i].large])
    large = np.array([1e3 * lat[i] for i in done if trace[i].large])
    served_evals = sum(instance_evals(trace[i].spec.n, trace[i].spec.k) for i in done)
    offered_evals = sum(instance_evals(r.spec.n, r.spec.k) for r in trace)

    def pct(a, p):
        return float(np.percentile(a, p)) if a.size else None

    line = {"metric": "serve p99 ms", "value": pct(lat_ms, 99), "unit": "ms", "n_gpus": 1, "steps": 1,
            "warmup": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
            "data": "synthetic (seeded Poisson request trace)",
            "config": {"workload": f"serving: Poisson {args.rate}/s over {args.horizon}s, "
                                   f"{100 * args.large_frac:.0f}% large (n={args.large_n}, d=32), rest GMM instance mix",
                       "slots": args.slots, "budget_gb": args.budget_gb, "large_threshold": args.large_threshold,
                       "large_ctas": args.large_ctas, "max_large": args.max_large, "drain_s": args.drain,
                       "greedy": "full rounds" if args.no_lazy else f"lazy rounds (same picks) for n >= {args.lazy_min_n}",
                       "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
                       "host_generation_s": gen_s},
            "latency_ms": {"p50": pct(lat_ms, 50), "p90": pct(lat_ms, 90), "p99": pct(lat_ms, 99),
                           "max": float(lat_ms.max()) if lat_ms.size else None,
                           "small_p50": pct(small, 50), "small_p99": pct(small, 99),
                           "large_p50": pct(large, 50), "large_p99": pct(large, 99)},
            "requests": {"offered": len(trace), "completed": len(done), "unfinished": len(trace) - len(done),
                         "large_offered": sum(r.large for r in trace), "large_completed": int(large.size)},
            "throughput": {"requests_per_s": len(done) / wall,
                           "full_round_equivalent_evals_per_s": served_evals / wall,
                           "performed_evals_per_s": st["evals_performed"] / wall,
                           "offered_full_round_equivalent_evals_per_s": offered_evals / args.horizon,
                           "offered_requests_per_s": len(trace) / args.horizon,
                           "wall_s": wall,
                           "note": "full-round equivalent counts sum_t (n - t) n per served request; lazy rounds "
                                   "(large requests) evaluate far fewer pairs, counted in performed_evals_per_s"},
            "saturation": {"saturated": len(done) < len(trace) or wall > 1.1 * args.horizon,
                           "drain_s": wall - args.horizon,
                           "served_requests_per_s": len(done) / wall},
            "batch_stats": st, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_sets(args):
    """Multi-set evaluation: n=50,000, d=64, 1,024 CSR sets of size U{1..64}
    (32-cluster anisotropic GMM).  One step = one ebc_eval_sets call over all
    sets; one evaluation = one (point, member) pair, n * nnz per step.  The
    tensor-core precision is timed against the FP32 plain kernel on the same
    handle; raw error against the oracle on a sample of sets."""
    import torch

    import oracle
    from paper_2105_12026_gb300 import ebc, synth
    torch.cuda.set_device(0)
    w = synth.multiset_eval(seed=args.seed, n=args.n, d=args.d, l=args.sets)
    V, idx, off = w["V"], w["idx"], w["off"]
    n, d = V.shape
    l = len(off) - 1
    nnz = int(off[-1])
    evals = n * nnz
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", 0)
    Vd = torch.from_numpy(V).to(dev)
    idx_d = torch.from_numpy(idx).to(dev)
    off_d = torch.from_numpy(off).to(dev)
    out = torch.empty(l, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    inst = ebc.Instance(Vd, precision=args.prec, stream=stream)

    def timed(prec):
        inst.set_precision(prec)
        if prec != "fp32":
            inst.reserve_sets(l, nnz)  # calls read nothing back to the host
        for _ in range(args.warmup):
            ebc.ebc_eval_sets(inst.h, idx_d.data_ptr(), off_d.data_ptr(), l, out.data_ptr())
        inst.sync()
        inst.profiling(True)
        inst.reset_profile()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for s in range(args.steps):
            flush.zero_()
            ev[s][0].record(stream)
            ebc.ebc_eval_sets(inst.h, idx_d.data_ptr(), off_d.data_ptr(), l, out.data_ptr())
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        inst.sync()
        prof = inst.profile()
        inst.profiling(False)
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        return ms, prof, out.cpu().numpy().copy()

    clocks = ClockSampler(0)
    clocks.start()
    ms_tc, prof_tc, f_tc = timed(args.prec)
    clk = clocks.stop()
    ms_32, prof_32, f_32 = timed("fp32")
    # e2e: host buffers through the C ABI (offsets, members in; values out)
    inst.set_precision(args.prec)
    inst.eval_sets_host(idx, off)
    e2e = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        inst.eval_sets_host(idx, off)
        e2e.append(time.perf_counter() - t0)
    inst.close()
    pick = np.random.default_rng(0).choice(l, min(48, l), replace=False)
    sub_off = np.zeros(pick.size + 1, np.int64)
    sub_off[1:] = np.cumsum(off[pick + 1] - off[pick])
    sub_idx = np.concatenate([idx[off[j]:off[j + 1]] for j in pick]).astype(np.int32)
    t0 = time.perf_counter()
    ref = oracle.eval_sets(V, sub_idx, sub_off)
    cpu_s = time.perf_counter() - t0
    rel_tc = np.abs(f_tc[pick] - ref) / np.maximum(ref, 1e-300)
    rel_32 = np.abs(f_32[pick] - ref) / np.maximum(ref, 1e-300)
    pk = peaks()
    kern_ms = prof_tc["eval_ms"] / max(1, args.steps)
    flops = 2.0 * d * evals
    achieved = flops / (kern_ms / 1e3) / 1e12 if kern_ms > 0 else None
    peak = pk["bf16"]
    line = {"metric": METRIC, "value": evals / (ms_tc / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_tc, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"bf16": "bf16", "fp16": "f16", "fp32": "f32"}.get(args.prec, args.prec),
            "data": "synthetic (seeded 32-cluster anisotropic GMM, CSR sets U{1..64})",
            "config": {"workload": f"multi-set evaluation n={n} d={d} l={l} sets of size U{{1..64}} (nnz={nnz})",
                       "l2": "flushed between calls (256 MB write, outside the events)",
                       "evals_per_step": evals},
            "roofline": {"bound": "tensor", "unit": "TFLOP/s", "achieved": achieved, "peak": peak,
                         "frac": achieved / peak if achieved else None, "traffic": None,
                         "peak_source": f"{pk['source']} bf16 burst",
                         "kernel": "multi-set evaluation (device plan + member gather + tcgen05 sets kernel "
                                   "+ finalize)",
                         "avg_ms": kern_ms, "algorithmic_flops_per_launch": flops},
            "gpu_launches": prof_tc["launches"], "clocks": clk,
            "fp32_plain": {"value": evals / (ms_32 / 1e3), "unit": UNIT, "ms_per_step": ms_32,
                           "tc_over_fp32": ms_32 / ms_tc},
            "raw_rel_err_vs_oracle": {"tc_max": float(rel_tc.max()), "tc_median": float(np.median(rel_tc)),
                                      "fp32_max": float(rel_32.max()), "sets_checked": int(pick.size),
                                      "tc_per_set": {str(int(j)): float(r) for j, r in zip(pick, rel_tc)}},
            "e2e": {"value": evals * args.steps / sum(e2e), "unit": UNIT,
                    "h2d_bytes_per_step": int(idx.nbytes + off.nbytes), "d2h_bytes_per_step": int(l * 8)},
            "cpu_baseline": {"value": n * int(sub_off[-1]) / cpu_s, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": f"oracle eval_sets on {pick.size} sampled sets "
                                                         f"({int(sub_off[-1])} members) x {n} points, {cpu_s:.1f}s"}}
    print(json.dumps(line), flush=True)
    return 0


def run_sieve(args):
    """Three Sieves (the streaming optimiser of the paper's case study, Sec. 6
    Fig. 4; rule of Sec. 2 / Sec. 4.1) over the drifting-regime features,
    stream in time order.  One step = reset to S = {} + one pass of the
    threshold sieve over the whole stream (ebc_sieve_host: bulk tensor-core
    upper bounds of each batch, exact gains of the items that may pass).
    Metric: distance evaluations per second, one evaluation being one
    (streamed item, point) pair bounded or evaluated exactly.  The largest
    singleton value m (an input of Three Sieves) is computed once, untimed."""
    import torch

    import oracle
    from paper_2105_12026_gb300 import ebc, synth
    torch.cuda.set_device(0)
    n, d, K = args.n, args.d, args.k
    eps, T = args.sieve_eps, args.sieve_patience
    V = synth.regime_greedy(seed=args.seed, n=n, d=d, k=K)["V"]
    stream = np.arange(n, dtype=np.int32)
    dev = torch.device("cuda", 0)
    cstream = torch.cuda.current_stream()
    Vd = torch.from_numpy(V).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    inst = ebc.Instance(Vd, precision=args.prec, stream=cstream)
    m1 = inst.max_singleton()
    thr = ebc.ebc_threshold_ladder(m1, K, eps, 1.0)

    def one_pass():
        inst.reset()
        sv = inst.sieve(K, thr, T)
        idx, f = sv.feed(stream)
        return idx, f, sv.counters()

    for _ in range(args.warmup):
        one_pass()
    torch.cuda.synchronize()
    inst.profiling(True)
    inst.reset_profile()
    clocks = ClockSampler(0)
    clocks.start()
    ms, evs, res = [], 0, None
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cstream)
        idx, f, cnt = one_pass()
        b.record(cstream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        evs += (cnt["bounded"] + cnt["exact"]) * n
        res = (idx, f, cnt)
    clk = clocks.stop()
    prof = inst.profile()
    inst.profiling(False)
    idx, f, cnt = res
    tot_ms = sum(ms)
    # primed: the pass starts from the singleton bounds (one bulk pass at
    # S = {}, inside the timed region), which reject most items without work
    pr_ms, pr_cnt = [], None
    for w in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cstream)
        inst.reset()
        sv = inst.sieve(K, thr, T, bounds=inst.gain_bounds_host())
        pidx, pf = sv.feed(stream)
        b.record(cstream)
        torch.cuda.synchronize()
        if w >= args.warmup:
            pr_ms.append(a.elapsed_time(b))
            pr_cnt = sv.counters()
    assert pidx.tolist() == idx.tolist() and np.array_equal(pf, f), "primed pass changed a decision"
    # e2e: V from pinned host memory into the handle, the stream from host
    # memory, accepted items and f back to the host, all inside the region
    e2e = []
    if not args.no_e2e:
        Vh = torch.from_numpy(V).pin_memory()
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            inst.reload(Vh)
            one_pass()
            e2e.append(time.perf_counter() - t0)
    # Sieve Streaming (one sieve per threshold up to 2 K m, eps = 0.1) on 8
    # instances at once, wall clock after one untimed run
    ss_eps, ss_workers = 0.1, args.ss_workers
    if ss_workers > 0:
        ebc.sieve_streaming(inst, stream, K, ss_eps, m1, workers=ss_workers, V=Vd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ss_idx, ss_f, ss_ends, ss_thr = ebc.sieve_streaming(inst, stream, K, ss_eps, m1, workers=ss_workers, V=Vd)
        torch.cuda.synchronize()
        ss_s = time.perf_counter() - t0
    # Greedy at the same K, for the quality context (lazy rounds, untimed here)
    inst.reset()
    inst.set_lazy(True)
    g_idx, g_f = inst.greedy_host(K)
    inst.close()
    pk = peaks()
    list_ms = prof["list_ms"] / max(1, args.steps)
    bulk_evals = cnt["bounded"] * n
    flops = 2.0 * d * bulk_evals
    achieved = flops / (list_ms / 1e3) / 1e12 if list_ms > 0 else None
    peak = pk["bf16_sustained"]
    line = {"metric": METRIC, "value": evs / (tot_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"bf16": "bf16", "fp16": "f16", "fp32": "f32"}.get(args.prec, args.prec),
            "data": "synthetic (seeded generator, drifting-regime injection-moulding-like features)",
            "config": {"workload": f"Three Sieves over the drifting-regime features n={n} d={d} K={K} eps={eps} "
                                   f"T={T}, stream in time order",
                       "precision": args.prec, "thresholds": int(thr.size), "m_single": m1,
                       "l2": "flushed between steps (256 MB write)",
                       "evals_per_step": evs // args.steps,
                       "timing": "CUDA events around the host-driven pass (it synchronises per batch)"},
            "roofline": {"bound": "tensor", "unit": "TFLOP/s", "achieved": achieved, "peak": peak,
                         "frac": achieved / peak if achieved else None, "traffic": None,
                         "peak_source": f"{pk['source']} bf16 sustained",
                         "kernel": "bulk bounds of the streamed batches (gather + tcgen05 gains kernel)",
                         "avg_ms": list_ms, "algorithmic_flops_per_launch": flops / max(1, prof["list_launches"]
                                                                                      // max(1, args.steps))},
            "gpu_launches": prof["launches"] // max(1, args.steps), "clocks": clk,
            "sieve": {"accepted": int(idx.size), "f_final": float(f[-1]) if f.size else 0.0,
                      "consumed": int(cnt["consumed"]), "bounded_items": int(cnt["bounded"]),
                      "exact_items": int(cnt["exact"]), "final_level": int(cnt["level"]),
                      "items_per_s": n / (tot_ms / args.steps / 1e3),
                      "ms_bulk_bounds": list_ms, "ms_exact": prof["refine_ms"] / max(1, args.steps),
                      "primed": {"ms_per_pass": sum(pr_ms) / len(pr_ms), "bounded_items": int(pr_cnt["bounded"]),
                                 "exact_items": int(pr_cnt["exact"]),
                                 "note": "includes the singleton bounds (one bulk pass at S = {}); same decisions"}},
            "sieve_streaming": {"eps": ss_eps, "sieves": int(ss_thr.size), "workers": ss_workers,
                                "wall_ms": 1e3 * ss_s, "f_best": max(ss_ends),
                                "ratio_over_greedy": max(ss_ends) / float(g_f[-1]),
                                "timing": "wall clock incl. creating the worker instances"} if ss_workers > 0 else None,
            "greedy_same_K": {"f_final": float(g_f[-1]), "ratio_sieve_over_greedy":
                              (float(f[-1]) / float(g_f[-1])) if f.size else 0.0},
            "e2e": {"value": evs / args.steps * len(e2e) / sum(e2e), "unit": UNIT,
                    "h2d_bytes_per_step": int(V.nbytes + stream.nbytes),
                    "d2h_bytes_per_step": int(idx.size * 12)} if e2e else None}
    if not args.no_cpu_baseline:
        m = oracle.norms(V)
        t0 = time.perf_counter()
        oracle.gains(V, m, [0])
        per_item = max(time.perf_counter() - t0, 1e-4)
        L = int(max(8, min(n, args.cpu_budget / per_item)))
        t0 = time.perf_counter()
        r = oracle.sieve(V, stream[:L], K, thr, T)
        cpu_s = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": L * n / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"oracle Three Sieves over the first {L} stream items "
                                          f"({r['idx'].size} accepted), {cpu_s:.1f}s, one item at a time"}
    print(json.dumps(line), flush=True)
    return 0


def run_sets_sweep(args):
    """Multi-set evaluation over the grid of the paper's runtime study (Sec. 5,
    Fig. 2 shape: d = 100, defaults N = 50,000, l = 5,000 sets of k = 10
    members, each of N, l, k varied), FP32 plain vs BF16 tensor cores.
    Synthetic GMM points and uniform random sets."""
    import torch

    from paper_2105_12026_gb300 import ebc, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    d = 100
    grid = [(50_000, 5_000, 10)]
    grid += [(N, 5_000, 10) for N in (1_000, 10_000, 100_000, 400_000)]
    grid += [(50_000, l, 10) for l in (1_000, 26_070)]
    grid += [(50_000, 5_000, k) for k in (100, 430)]
    rows = []
    for (N, l, k) in grid:
        rng = np.random.default_rng(args.seed + N + l + k)
        V = synth.zscore_to_f32(synth.gaussian_mixture(rng, N, d, 32, sigma=None))
        idx, off = synth.random_sets(rng, N, l, k, k)
        Vd = torch.from_numpy(V).to(dev)
        idx_d, off_d = torch.from_numpy(idx).to(dev), torch.from_numpy(off).to(dev)
        out = torch.empty(l, dtype=torch.float64, device=dev)
        inst = ebc.Instance(Vd, stream=stream)
        row = {"N": N, "l": l, "k": k, "pairs": N * int(off[-1])}
        for prec in ("fp32", "bf16"):
            inst.set_precision(prec)
            ebc.ebc_eval_sets(inst.h, idx_d.data_ptr(), off_d.data_ptr(), l, out.data_ptr())
            inst.sync()
            ms = []
            for _ in range(max(1, args.steps)):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ebc.ebc_eval_sets(inst.h, idx_d.data_ptr(), off_d.data_ptr(), l, out.data_ptr())
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            inst.sync()
            row[prec + "_ms"] = min(ms)
            row[prec + "_pairs_per_s"] = row["pairs"] / (min(ms) / 1e3)
        row["bf16_over_fp32"] = row["fp32_ms"] / row["bf16_ms"]
        inst.close()
        rows.append(row)
        del Vd, idx_d, off_d, out
    base = rows[0]
    line = {"metric": METRIC, "value": base["bf16_pairs_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": 1, "ms_per_step": base["bf16_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic (32-cluster GMM, z-scored; uniform random sets)",
            "config": {"workload": "multi-set evaluation sweep, d=100 (N, l, k grid around N=50,000 l=5,000 k=10)",
                       "l2": "flushed between calls"},
            "sweep": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_case_study(args):
    """The shape of the paper's case-study timing (Sec. 6, Fig. 4: summaries
    of size K from n = 1,000 cycles of d = 3,524 samples by Greedy and by
    Three Sieves), on synthetic sensor curves (`synth.case_study_series`).
    Per K: BF16 Greedy (full and lazy rounds; the K-blocked tensor-core bulk
    kernel), FP32 plain Greedy, and Three Sieves (eps = 0.1, T = 10) over
    the cycles in time order; device time with CUDA events.  Metric: Greedy's
    distance evaluations per second at the largest K."""
    import torch

    import oracle
    from paper_2105_12026_gb300 import ebc, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", 0)
    n, d = 1_000, 3_524
    V = synth.case_study_series(seed=args.seed, n=n, d=d)
    Vd = torch.from_numpy(V).to(dev)
    items = np.arange(n, dtype=np.int32)
    Ks = (10, 20, 50, 100, 200)

    def timed(fn):
        fn()  # warm-up (also sets kernel attributes and captures graphs)
        best = None
        for _ in range(max(1, args.steps)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        return best, out

    rows = []
    clocks = ClockSampler(0)
    clocks.start()
    with ebc.Instance(Vd, precision="bf16", stream=stream) as g16, \
            ebc.Instance(Vd, precision="bf16", stream=stream, lazy=True) as gl, \
            ebc.Instance(Vd, precision="fp32", stream=stream) as g32:
        m1 = g16.max_singleton()
        for K in Ks:
            def greedy(inst):
                inst.reset()
                return inst.greedy_host(K)
            ms16, (i16, f16) = timed(lambda: greedy(g16))
            msl, (il, fl) = timed(lambda: greedy(gl))
            ms32, (i32, f32) = timed(lambda: greedy(g32))

            def sieve():
                g16.reset()
                return ebc.three_sieves(g16, items, K, 0.1, 10, m1)
            mss, (isv, fsv, _) = timed(sieve)
            rows.append({"K": K, "greedy_bf16_ms": ms16, "greedy_lazy_ms": msl, "greedy_fp32_ms": ms32,
                         "three_sieves_ms": mss, "greedy_f": float(f16[-1]),
                         "three_sieves_f": float(fsv[-1]) if fsv.size else 0.0, "three_sieves_size": int(isv.size),
                         "picks_equal_fp32": bool(np.array_equal(i16, i32)), "lazy_equal": bool(np.array_equal(i16, il))})
    clk = clocks.stop()
    last = rows[-1]
    evals = sum((n - t) * n for t in range(last["K"]))
    t0 = time.perf_counter()
    oracle.greedy(V, 2)
    cpu_s = time.perf_counter() - t0
    line = {"metric": METRIC, "value": evals / (last["greedy_bf16_ms"] / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": 1, "ms_per_step": last["greedy_bf16_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic sensor curves (8 regimes of sinusoid templates + noise, z-scored)",
            "config": {"workload": f"case-study shape: n={n} cycles of d={d} samples, summaries K in {list(Ks)}",
                       "evals_per_step": evals, "l2": "not flushed (the 14 MB instance is L2-resident by design)"},
            "case_study": rows, "clocks": clk,
            "cpu_baseline": {"value": 2 * n * n / cpu_s, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"oracle Greedy k=2 on the same instance, FP64, {cpu_s:.1f}s"}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    if any(w in sys.argv for w in ("mix", "serve")):
        # many instance streams: give them their own hardware queues (read at
        # the first CUDA call, which has not happened yet)
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp16", "fp8", "fp32"])
    ap.add_argument("--refine-k", type=int, default=8)
    ap.add_argument("--workload", default="regime", choices=["regime", "small", "mix", "serve", "sets", "sets-sweep", "sieve", "case-study"])
    ap.add_argument("--sets", type=int, default=1024, help="sets: number of CSR sets")
    ap.add_argument("--instances", type=int, default=256, help="mix: number of instances")
    ap.add_argument("--mix-mode", default="group", choices=["group", "streams", "batch"],
                    help="mix: one shared bulk launch per round (group), per-instance rounds on own streams "
                         "(streams) or the batch runtime (batch)")
    ap.add_argument("--group-lanes", type=int, default=1, help="mix: lanes of the shared-launch group")
    ap.add_argument("--group-by-width", action="store_true", help="mix: group lanes by row width")
    ap.add_argument("--group-ctas", type=int, default=0, help="mix: CTA cap of the shared launch (0: all SMs)")
    ap.add_argument("--slots", type=int, default=32, help="mix/serve: concurrent instances")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="mix/serve: device-memory budget")
    ap.add_argument("--rate", type=float, default=50.0, help="serve: arrivals per second")
    ap.add_argument("--horizon", type=float, default=10.0, help="serve: arrival horizon in seconds")
    ap.add_argument("--drain", type=float, default=60.0, help="serve: seconds allowed after the horizon")
    ap.add_argument("--large-frac", type=float, default=0.05, help="serve: fraction of large requests")
    ap.add_argument("--large-n", type=int, default=1_000_000, help="serve: n of large requests")
    ap.add_argument("--large-threshold", type=int, default=500_000, help="serve: n from which the CTA cap applies")
    ap.add_argument("--large-ctas", type=int, default=120, help="serve: CTA cap of large requests (0 = none)")
    ap.add_argument("--max-large", type=int, default=2, help="serve: large requests running at once (0 = any)")
    ap.add_argument("--sieve-eps", type=float, default=0.01, help="sieve: threshold ladder step")
    ap.add_argument("--sieve-patience", type=int, default=1000, help="sieve: Three Sieves T")
    ap.add_argument("--ss-workers", type=int, default=8, help="sieve: instances running Sieve Streaming (0: skip)")
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--d", type=int, default=128)
    ap.add_argument("--k", type=int, default=100)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp8-peak", action="store_true", help="fp8: skip measuring the FP8 GEMM peak")
    ap.add_argument("--no-raw-error", action="store_true", help="skip the raw low-precision gain error sample")
    ap.add_argument("--no-lazy", action="store_true", help="regime: skip the lazy comparison; serve: full rounds")
    ap.add_argument("--lazy-min-n", type=int, default=100_000, help="serve: lazy rounds from this n")
    ap.add_argument("--greedy", default="full", choices=["full", "lazy"], help="regime/small: round kind timed")
    ap.add_argument("--autotune", type=int, default=0, help="regime/small: autotune the bulk kernel first (reps)")
    ap.add_argument("--tune-file", default="", help="save the tuning table here after autotuning")
    ap.add_argument("--fp32-rounds", type=int, default=3, help="rounds of the FP32 plain comparison")
    ap.add_argument("--ref-cands", type=int, default=64, help="reference arm: candidates per step")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "mix":
        return run_mix(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "sets-sweep":
        return run_sets_sweep(args)
    if args.workload == "sieve":
        return run_sieve(args)
    if args.workload == "case-study":
        return run_case_study(args)
    if args.workload == "sets":
        if args.n == 200_000 and args.d == 128:
            args.n, args.d = 50_000, 64
        return run_sets(args)

    import torch
    import torch.distributed as dist

    from paper_2105_12026_gb300 import build as _b
    from paper_2105_12026_gb300 import ebc

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if not os.path.exists(_b.LIB):
        raise SystemExit("CUDA library not built; run __graft_entry__.build() first")

    def barrier():
        if world > 1:
            dist.barrier()

    V, k, wname = make_workload(args, rank)
    n, d = V.shape
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    Vd = torch.from_numpy(V).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    lazy_main = args.greedy == "lazy" and args.prec != "fp32"
    inst = ebc.Instance(Vd, precision=args.prec, refine_k=args.refine_k, stream=stream, lazy=lazy_main)
    tuned = None
    if args.autotune > 0 and args.prec != "fp32":
        t0 = time.perf_counter()
        inst.autotune(args.autotune)  # outside the timed region; results do not depend on it
        tuned = {"reps": args.autotune, "search_s": time.perf_counter() - t0, "entry": inst.tune_entry()}
        if args.tune_file:
            ebc.ebc_tune_save(args.tune_file)
    out_idx = torch.empty(k, dtype=torch.int32, device=dev)
    out_f = torch.empty(k, dtype=torch.float64, device=dev)

    def step():
        inst.reload(Vd)
        ebc.ebc_greedy(inst.h, k, out_idx.data_ptr(), out_f.data_ptr())

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    inst.sync()

    # timed region -------------------------------------------------------
    inst.profiling(True)
    inst.reset_profile()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()  # L2 flush, outside the step's events
        ev[s][0].record(stream)
        step()
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    prof = inst.profile()
    inst.profiling(False)
    inst.sync()
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    idx_bf = out_idx.cpu().numpy().copy()
    f_bf = out_f.cpu().numpy().copy()
    stats = inst.stats()

    t_max_ms = max_over_ranks(dev_ms, world, dev)
    evals_step = greedy_evals(n, k)
    if lazy_main:
        # lazy rounds: the evaluations actually performed (bulk candidates x n)
        evals_step = stats["bulk_candidates"] * n  # reload resets the counters: the last step's
    value = world * args.steps * evals_step / (t_max_ms / 1e3)

    # roofline of the dominant kernel (the bulk gains kernel) -------------
    pk = peaks()
    bulk_avg_s = prof["bulk_ms"] / 1e3 / max(1, prof["bulk_launches"])
    evals_per_launch = prof["bulk_evals"] / max(1, prof["bulk_launches"])
    if lazy_main:
        # a lazy round launches the row gather and the bulk kernel of its list under one timer
        evals_per_launch = stats["bulk_candidates"] * n * args.steps / max(1, prof["list_launches"] // 2)
        bulk_avg_s = prof["list_ms"] / 1e3 / max(1, prof["list_launches"] // 2)
    if args.prec == "fp32":
        # direct (v - c)^2: sub + fma per (pair, dim) = 3 flops, 2 lane-ops;
        # 152 SMs x 128 FP32 lanes at the maximum SM clock
        flops = 3.0 * d * evals_per_launch
        peak = 152 * 128 * 1.5 * pk["sm_max_mhz"] * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak_source": "derived: 152 SM x 128 FP32 lanes x 1.5 flop/lane-op "
                                                                   "x max SM clock"}
    else:
        flops = 2.0 * d * evals_per_launch
        peak = pk["bf16_sustained"]
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak_source": f"{pk['source']} bf16 sustained"}
        if args.prec == "fp8":
            fp8 = measure_fp8_peak() if not args.no_fp8_peak else {"sustained": None, "how": "not measured"}
            if fp8["sustained"]:
                peak = fp8["sustained"]
                roof["peak_source"] = "measured fp8 sustained in this run (" + fp8["how"] + ")"
                roof["fp8_peak_burst"] = fp8["burst"]
            else:
                peak = 2 * pk["bf16_sustained"]
                roof["peak_source"] = f"{pk['source']} bf16 sustained x2 (fp8 nominal ratio; {fp8['how']})"
    achieved = flops / bulk_avg_s / 1e12 if bulk_avg_s > 0 else None
    roof.update({"achieved": achieved, "peak": peak, "frac": (achieved / peak) if achieved else None,
                 "traffic": None if lazy_main else NCU_TRAFFIC.get((args.prec, n, d)), "traffic_unit": "bytes per launch (ncu)", "kernel": "bulk gains", "launches": prof["bulk_launches"],
                 "avg_ms": bulk_avg_s * 1e3, "algorithmic_flops_per_launch": flops})

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16",
                                                              "fp8": "fp8e4m3"}[args.prec],
            "data": "synthetic (seeded generator, drifting-regime injection-moulding-like features)",
            "config": {"workload": wname + (" (lazy rounds)" if lazy_main else ""), "n": n, "d": d, "k": k,
                       "precision": args.prec, "refine_k": args.refine_k,
                       "greedy": "lazy rounds: value counts the evaluations performed" if lazy_main else "full rounds",
                       "autotune": tuned,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "flushed between steps (256 MB write, outside the step events)",
                       "evals_per_step": evals_step, "wall_s_timed_region": t_wall},
            "roofline": roof, "gpu_launches": prof["launches"], "clocks": clk,
            "certification": {k2: stats[k2] for k2 in ("rounds", "certified_rounds", "escalated_rounds",
                                                         "escalated_candidates", "max_raw_rel_err")},
            "breakdown_ms_per_step": {"bulk_gains": prof["bulk_ms"] / args.steps,
                                      "list_bounds": prof["list_ms"] / args.steps,
                                      "exact_refine": prof["refine_ms"] / args.steps,
                                      "rest": t_max_ms / args.steps
                                      - (prof["bulk_ms"] + prof["list_ms"] + prof["refine_ms"]) / args.steps},
            "f_final": float(f_bf[-1]), "picks_head": idx_bf[:10].tolist()}

    # FP32 plain comparison at matched picks ------------------------------
    if args.prec != "fp32" and args.fp32_rounds > 0 and rank == 0:
        R = min(args.fp32_rounds, k)
        p32 = ebc.Instance(Vd, precision="fp32", stream=stream)
        p32.greedy(R)  # warm
        p32.reload(Vd)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        i32, f32 = p32.greedy(R)
        b.record(stream)
        torch.cuda.synchronize()
        ms32 = a.elapsed_time(b)
        ev32 = greedy_evals(n, R)
        i32 = i32.cpu().numpy()
        p32.close()
        v32 = ev32 / (ms32 / 1e3)
        line["fp32_plain"] = {"value": v32, "unit": UNIT, "rounds": R,
                              "picks_match": bool((i32 == idx_bf[:R]).all()),
                              "tc_over_fp32": value / world / v32}

    # lazy Greedy on the same workload (same picks, fewer bulk candidates) --
    if args.prec != "fp32" and not args.no_lazy and not lazy_main and rank == 0:
        lz = ebc.Instance(Vd, precision=args.prec, refine_k=args.refine_k, stream=stream, lazy=True)
        lz.greedy(k)  # warm (graph capture)
        torch.cuda.synchronize()
        lev = []
        for s in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lz.reload(Vd)
            il, fl = lz.greedy(k)
            b.record(stream)
            lev.append((a, b))
        torch.cuda.synchronize()
        lms = sum(a.elapsed_time(b) for a, b in lev) / args.steps
        lst = lz.stats()
        lz.close()
        line["lazy"] = {"ms_per_step": lms, "speedup_vs_full": (t_max_ms / args.steps) / lms,
                        "bulk_candidates_per_step": lst["bulk_candidates"],
                        "full_candidates_per_step": sum(n - t for t in range(k)),
                        "picks_match_full": bool((il.cpu().numpy() == idx_bf).all()),
                        "f_match_full": bool((fl.cpu().numpy() == f_bf).all())}

    # end-to-end through the C ABI with host buffers ----------------------
    if not args.no_e2e:
        Vh = torch.from_numpy(V).pin_memory()
        for _ in range(1):
            inst.reload(Vh)
            inst.greedy_host(k)
        e2e_t = []
        barrier()
        for s in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            inst.reload(Vh)  # host -> device copy of V inside the step
            hidx, hf = inst.greedy_host(k)  # device -> host read of the picks and f
            e2e_t.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(sum(e2e_t), world, dev)
        line["e2e"] = {"value": world * args.steps * evals_step / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": int(n * d * 4), "d2h_bytes_per_step": int(k * (4 + 8))}

    if rank == 0 and args.prec != "fp32" and not args.no_raw_error:
        # raw low-precision gains (no certification) of a seeded sample of
        # candidates at S = {}, against the FP64 oracle, per result
        import oracle
        inst.reset()
        samp = np.sort(np.random.default_rng(args.seed + 7).choice(n, 64, replace=False)).astype(np.int32)
        raw = inst.gains_host(samp)
        ref = oracle.gains(V, oracle.norms(V), samp)
        rel = np.abs(raw - ref) / np.maximum(np.abs(ref), 1e-300)
        line["raw_rel_err_vs_oracle"] = {"what": "ebc_gains at S = {} (raw, uncertified) vs FP64 oracle",
                                         "max": float(rel.max()), "median": float(np.median(rel)),
                                         "p90": float(np.percentile(rel, 90)),
                                         "per_candidate": {str(int(c)): float(r) for c, r in zip(samp, rel)}}
    inst.close()
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(V, args.cpu_budget)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
