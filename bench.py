#!/usr/bin/env python3
"""Benchmark of the dense ternary prime-implicant sweep (DenseQMC, arXiv 2302.10083).

Workload: one n = 24 function, ON ~ Bernoulli(0.85) (seed 1 + rank), no
don't-cares: 3^24 = 2.82e11 cubes.  One step = the whole hot path on the
device: every sweep pass (truth table -> Merge -> fused Merge/Reduce ->
Reduce -> dense prime bitmap + count) and the compaction of the bitmap into the
(mask, value) list, with the truth table already in HBM.  The state (37 GB)
and bitmap (35 GB) are far larger than the 129 MB L2, so no L2 flush is done
between steps.

Prints one JSON line (rank 0).  With --gpus N under torchrun every rank sweeps
its own function (replicas, weak scaling; the passes need no exchange).

--impl reference times the CPU oracle (plain C, Algorithm 3, one byte per
cube, OpenMP on the host cores) on a bounded sample of the same workload
family: the same generator and density at n = 19 per step.

--workload serving (not the default line): Poisson arrivals at 1e2, 1e3, 1e4
and 1e5 jobs/s of functions with n log-uniform in 6..22 and ON density
uniform in [0.2, 0.95], replayed against the library's serving loop
(continuous batching, admission by device-memory footprint) and against the
same loop run one job at a time; p50/p99 latency (arrival to result) and
jobs/s for both, and the two must give the same prime counts.

--workload batched (not the default line): 65,536 independent functions, n
uniform in 4..14, ON density uniform in [0.3, 0.9], 10% with a Bernoulli(0.05)
don't-care set.  It times the batch as one CUDA-graph launch (dqmc_batch_run)
and as one dqmc_primes_dev call per function, checks that both give the same
bitmaps and counts, and prints functions/s for each.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_MAIN = 24
P_ON = 0.85
REF_SAMPLE_N = 19       # --impl reference: one oracle sweep of this size per step
CPU_BASELINE_N = 20     # cpu_baseline: one oracle sweep of this size
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0   # GB300 HBM3e, nominal (about 8 TB/s)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_MAIN)
    ap.add_argument("--p-on", type=float, default=P_ON,
                    help="single workload: ON density (the workload's is 0.85; 1.0 = constant 1)")
    ap.add_argument("--ref-n", type=int, default=REF_SAMPLE_N,
                    help="--impl reference: the n of the function the oracle sweeps per step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--inplace", action="store_true",
                    help="single workload: write the bitmap over the state (one array; n = 25 fits only so)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side", action="store_true",
                    help="single workload: leave out the compact batched and serving results of the line")
    ap.add_argument("--workload", choices=["single", "batched", "serving"], default="single")
    ap.add_argument("--serve-jobs", type=int, default=2000, help="serving: jobs per arrival rate at most")
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="serving: arrival span per rate at most")
    ap.add_argument("--batch", type=int, default=65536, help="functions in the batched workload")
    ap.add_argument("--batch-n", type=int, default=None,
                    help="batched: every function with this n (a one-class batch, for profiling one kernel)")
    ap.add_argument("--no-one-by-one", action="store_true",
                    help="batched: skip the one-launch-per-function comparison (for profiling the graph alone)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched: keep the built-in launch table instead of tuning it on the batch first")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device):
    """The largest x over all ranks (every rank gets it): a step time taken
    on each rank becomes the job's step time."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        sel = [p for (t, p) in self.samples if t0 <= t <= t1] or [p for (_, p) in self.samples[-5:]]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        sm = [float(p[1]) for p in sel if p[1].replace(".", "").isdigit()]
        smax = [float(p[2]) for p in sel if p[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in sel for i in range(4) if p[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(sel)}


# The sources the streaming pass kernels are compiled from: a change to any of
# them voids the stored ncu traffic of those kernels.
PASS_SOURCES = ("dqmc_api.cu", "dqmc_chunk.cuh", "dqmc_internal.h", "dqmc_pass.cu", "dqmc_steps.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2302_10083_gb300", "csrc")
    for name in PASS_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key, n):
    """dram read+write bytes of one launch of pass `kernel_key` at this n, from
    profiles/ncu_traffic.json, if that capture was taken at this n from the
    current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash() or d.get("n") != n:
        return None
    ent = d.get("passes", {}).get(kernel_key)
    return None if ent is None else ent["dram_read_bytes"] + ent["dram_write_bytes"]


def single_metric(n):
    """The metric string of the single-function line; the reference arm prints
    the same string so that the two lines can be compared."""
    return f"cubes/s (dense prime-implicant sweep, n={n} single function)"


def cpu_baseline(n=CPU_BASELINE_N):
    import oracle
    from paper_2302_10083_gb300 import synth
    on, _ = synth.random_function(n, 1, P_ON)
    t0 = time.perf_counter()
    oracle.sweep(n, on)
    dt = time.perf_counter() - t0
    cores = oracle.max_threads()
    # the same oracle on one thread, at a size that keeps it to a few seconds
    n1 = n - 3
    on1, _ = synth.random_function(n1, 1, P_ON)
    t1 = time.perf_counter()
    oracle.sweep(n1, on1, threads=1)
    dt1 = time.perf_counter() - t1
    return {"value": 3 ** n / dt, "unit": "cubes/s", "cores": cores, "kind": "oracle",
            "sample": f"one n={n} function of the same family (ON ~ Bernoulli({P_ON}), seed 1): full oracle "
                      f"sweep (Algorithm 3, one byte per cube, OpenMP), {dt:.2f} s; cubes/s = 3^{n}/time",
            "one_core": {"value": 3 ** n1 / dt1, "unit": "cubes/s", "cores": 1,
                         "sample": f"one n={n1} function of the same family, one thread, {dt1:.2f} s"}}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    from paper_2302_10083_gb300 import synth
    n = args.ref_n
    on, _ = synth.random_function(n, 1, P_ON)
    for _ in range(args.warmup):
        oracle.sweep(n, on)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sweep(n, on)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = 3 ** n / (ms / 1e3)
    line = {
        "impl": "reference", "metric": single_metric(N_MAIN), "value": value,
        "unit": "cubes/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"single function n={N_MAIN}, ON ~ Bernoulli({P_ON}); each reference step sweeps "
                               f"an n={n} function of the same family", "n": N_MAIN, "sample_n": n},
        "cpu_baseline": {"value": value, "unit": "cubes/s", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"n={n} oracle sweep per step (Algorithm 3, byte per cube)"},
        "e2e": {"value": value, "unit": "cubes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2302_10083_gb300 import dqmc, synth

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    n = args.n
    seed = 1 + rank
    p_on = args.p_on
    on, _ = synth.random_function(n, seed, p_on)
    L = dqmc.lib()
    # expected primes + 5% headroom sizes the list buffer
    from math import comb
    exp_primes = sum(comb(n, w) * 2 ** (n - w) * p_on ** (2 ** w) * (1 - p_on ** (2 ** w)) ** (n - w)
                     for w in range(n + 1))
    cap = int(exp_primes * 1.05) + 1024
    buf = dqmc.DeviceBuffers(n, device=f"cuda:{local}", with_dc=False, cap=cap, inplace=args.inplace)
    buf.on[: on.size].copy_(torch.from_numpy(on))
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    npass = dqmc.dqmc_plan_passes(n)
    plan = dqmc.dqmc_plan_json(n)
    def pass_name(i, q):
        ph = "+".join(f"{x['load']}" + ("M" if x["merge"] else "") + ("R" if x["reduce"] else "")
                      + ("c" if x["chunk_mask"] else "") + ("O" if x["out"] else "")
                      + f"[{x['a']}:{x['a'] + x['K']}|B{x['B']}]" for x in q["phases"])
        return f"pass{i}:{ph}"
    names = [pass_name(i, q) for i, q in enumerate(plan["passes"])]

    def step(events=None):
        for p in range(npass):
            st = L.dqmc_sweep_pass_dev(n, p, buf.on.data_ptr(), None, buf.bitmap.data_ptr(), buf.pairs.data_ptr(),
                                       cap, buf.count.data_ptr(), buf.work.data_ptr(), buf.work_bytes, sh)
            if st != 0:
                raise dqmc.DqmcError(st, f"pass {p}")
            if events is not None:
                events[p].record(stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    buf.status()
    count = int(buf.count.item())
    if count > cap:
        raise SystemExit(f"list overflow: {count} primes > cap {cap}")

    sampler = ClockSampler(local) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(npass)] for _ in range(K)]
    start = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    start.record(stream)
    for k in range(K):
        step(evs[k])
    torch.cuda.synchronize()
    barrier()
    t_wall1 = time.time()
    buf.status()  # raises DqmcError if a bounded device wait gave up
    count = int(buf.count.item())   # (also when no warm-up step ran)
    if count > cap:
        raise SystemExit(f"list overflow: {count} primes > cap {cap}")
    total_ms = start.elapsed_time(evs[K - 1][npass - 1])
    per_pass = [0.0] * npass
    for k in range(K):
        prev = start if k == 0 else evs[k - 1][npass - 1]
        for p in range(npass):
            per_pass[p] += prev.elapsed_time(evs[k][p]) if p == 0 else evs[k][p - 1].elapsed_time(evs[k][p])
    per_pass = [x / K for x in per_pass]
    ms = max_over_ranks(total_ms / K, world, f"cuda:{local}")
    clocks = None
    if sampler:
        time.sleep(0.3)
        sampler.stop()
        clocks = sampler.summary(t_wall0, t_wall1)

    cubes = 3 ** n
    value = world * cubes / (ms / 1e3)
    peak, peak_kind = measured_peaks()
    # dominant kernel = the sweep pass with the largest share of the step
    dom = max(range(npass), key=lambda p: per_pass[p])
    A = (cubes + 7) // 8
    b_roof = (1 << n) // 8 + 3 * A
    # The bitmap pass must read the merged state and write the primes: 2 A
    # bytes by the method (the padded rows and the list come on top; they are
    # the design bytes).
    dom_bytes = 2 * A if dom == npass - 1 else dqmc.dqmc_pass_bytes(n, dom, False)
    achieved = dom_bytes / (per_pass[dom] / 1e3) / 1e9
    passes = {}
    for p in range(npass):
        design = dqmc.dqmc_pass_bytes(n, p, False) + (8 * count if p == npass - 1 else 0)
        tr = ncu_traffic(f"pass{p}", n)
        passes[names[p]] = {"ms": per_pass[p], "design_bytes": design,
                            "design_gbs": design / (per_pass[p] / 1e3) / 1e9,
                            "traffic_bytes": tr,
                            "traffic_gbs": None if tr is None else tr / (per_pass[p] / 1e3) / 1e9}
    result = {
        "metric": single_metric(n),
        "value": value, "unit": "cubes/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 bitwise", "data": "synthetic",
        "config": {"workload": f"single function n={n}, ON ~ Bernoulli({p_on}), seed 1+rank, no don't-cares; "
                               f"step = full sweep + bitmap + count + (mask,value) list, inputs resident in HBM",
                   "n": n, "cubes": cubes, "primes": count, "l2": "no flush: state %.2f GB and bitmap %.2f GB >> 129 MB L2" % (
                       dqmc.dqmc_workspace_bytes(n) / 1e9, A / 1e9),
                   "bitmap": "written over the state (one array)" if args.inplace else "a buffer of its own",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic(f"pass{dom}", n),
                     "algorithmic_bytes_per_launch": dom_bytes,
                     "algorithmic_bytes_note": "the method's bytes: state read + primes written, 2*ceil(3^n/8) "
                                               "for the bitmap pass; padded rows and the list are in passes[].design_bytes"},
        "path_roofline": {"b_roof_bytes": b_roof, "achieved_gbs": b_roof / (ms / 1e3) / 1e9,
                          "frac_of_peak": b_roof / (ms / 1e3) / 1e9 / peak,
                          "frac_of_nominal": b_roof / (ms / 1e3) / 1e9 / NOMINAL_HBM_GBS,
                          "nominal_gbs": NOMINAL_HBM_GBS,
                          "note": "B_roof = 2^n/8 + 3*ceil(3^n/8): read input, write merged state, read it, write primes"},
        "per_kernel_ms": {names[p]: per_pass[p] for p in range(npass)},
        "passes": passes,
        "step_design_bytes": sum(x["design_bytes"] for x in passes.values()),
        "gpu_launches": K * npass,
        "clocks": clocks,
    }

    if not args.no_e2e:
        result["e2e"] = e2e_measure(args, n, on, cap, buf, dqmc, torch, K, world, local, barrier)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline()
    if world == 1 and not args.no_side:
        result["batched"] = batched_summary(args, local)
        result["serving"] = serving_summary(args, local)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def batched_summary(args, local):
    """The batched workload (65,536 functions) as a compact object of the main
    line: one graph launch per step (per-n kernels, and the same batch in one
    persistent launch) against one dqmc_primes_dev call per function, built-in
    launch table (the autotuner's choice on a GB300)."""
    a = argparse.Namespace(**vars(args))
    a.batch, a.batch_n, a.no_autotune, a.no_one_by_one, a.no_e2e = 65536, None, True, False, True
    a.steps, a.warmup = 10, 3
    r = run_batched(a, 0, 1, local, emit=False)
    return {"metric": r["metric"], "value": r["value"], "unit": r["unit"], "ms_per_step": r["ms_per_step"],
            "steps": a.steps, "one_launch_per_function": r["one_launch_per_function"],
            "speedup_vs_one_launch_per_function": r["speedup_vs_one_launch_per_function"],
            "results_identical": r["results_identical"], "cubes_per_s": r["cubes_per_s"],
            "one_persistent_launch": r["one_persistent_launch"],
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"], "config": r["config"]}


def serving_summary(args, local):
    """The serving workload at 1e4 and 1e5 arrivals/s (1000 jobs each) and
    the small-job stream (4000 jobs), continuous batching against one job at
    a time, as a compact object of the main line."""
    a = argparse.Namespace(**vars(args))
    a.serve_jobs = 1000
    r = run_serving(a, 0, 1, local, rates=[1e4, 1e5], emit=False)
    keep = ("jobs_per_s", "p50_ms", "p99_ms")
    rates = [{"rate_jobs_per_s": x["rate_jobs_per_s"], "jobs": x["jobs"],
              "continuous": {k: x["continuous"][k] for k in keep},
              "one_by_one": {k: x["one_by_one"][k] for k in keep},
              "throughput_speedup": x["throughput_speedup"], "p99_speedup": x["p99_speedup"],
              "counts_identical": x["counts_identical"]} for x in r["per_rate"]]
    sm = r["small_jobs"]
    small = {"jobs": sm["jobs"], "n": sm["n"], "rate_jobs_per_s": sm["rate_jobs_per_s"],
             "continuous": {k: sm["continuous"][k] for k in keep},
             "one_by_one": {k: sm["one_by_one"][k] for k in keep},
             "throughput_speedup": sm["throughput_speedup"], "counts_identical": sm["counts_identical"]}
    return {"metric": "served jobs/s, continuous batching vs one job at a time", "unit": "jobs/s",
            "per_rate": rates, "small_jobs": small, "config": r["config"]}


def e2e_measure(args, n, on, cap, buf, dqmc, torch, K, world, local, barrier):
    """Same metric through the host entry point dqmc_list: truth table from
    pinned host memory in, (mask, value) list and count out to pinned host
    memory, all inside the timed region."""
    import ctypes

    import numpy as np
    del buf
    torch.cuda.empty_cache()
    L = dqmc.lib()
    on_h = torch.from_numpy(np.ascontiguousarray(on)).pin_memory()
    out_h = torch.empty(2 * cap, dtype=torch.int32).pin_memory()
    cnt = ctypes.c_uint64()
    on_p = ctypes.cast(on_h.data_ptr(), dqmc.c_u8p)
    out_p = ctypes.cast(out_h.data_ptr(), dqmc.c_u32p)
    steps = max(1, min(K, 5))
    st = L.dqmc_list(n, on_p, None, out_p, cap, ctypes.byref(cnt))  # warm-up: device buffers allocated here
    if st != 0:
        raise dqmc.DqmcError(st, "dqmc_list")
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        st = L.dqmc_list(n, on_p, None, out_p, cap, ctypes.byref(cnt))
        if st != 0:
            raise dqmc.DqmcError(st, "dqmc_list")
    dt = max_over_ranks((time.perf_counter() - t0) / steps, world, f"cuda:{local}")
    dqmc.dqmc_release()
    return {"value": world * 3 ** n / dt, "unit": "cubes/s", "ms_per_step": 1e3 * dt, "steps": steps,
            "h2d_bytes_per_step": int(on.size), "d2h_bytes_per_step": int(8 * cnt.value + 8),
            "api": "dqmc_list (host buffers, pinned)"}


def run_batched(args, rank, world, local, emit=True):
    """Batched workload: one graph launch for the whole batch against one
    dqmc_primes_dev call per function, same device buffers.  Returns the
    result line (printed by rank 0 when emit)."""
    import numpy as np
    import torch

    from paper_2302_10083_gb300 import dqmc, synth

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    if args.batch_n is None:
        b = synth.batch_functions(count=args.batch, seed=1 + rank)
    else:
        b = synth.batch_functions(count=args.batch, seed=1 + rank, n_lo=args.batch_n, n_hi=args.batch_n)
    ns = b["n"].astype(np.uint32)
    nf = len(ns)
    arena_h = torch.from_numpy(b["arena"]).pin_memory()
    arena = arena_h.to(dev)
    bm_off, total = dqmc.batch_bitmap_layout(ns)
    bitmaps = torch.zeros(total, dtype=torch.uint8, device=dev)
    counts = torch.zeros(nf, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    L = dqmc.lib()

    def graph_run():
        st = dqmc.dqmc_batch_run(ns, b["tt_off"], arena.data_ptr(), b["dc_off"], counts.data_ptr(),
                                 bitmaps.data_ptr(), bm_off, sh)
        if st != 0:
            raise dqmc.DqmcError(st, "dqmc_batch_run")

    # autotuner (untimed): each n's launch shape, timed on this batch
    tune_s, tune_ms = None, None
    if not args.no_autotune:
        t_tune = time.perf_counter()
        tune_ms = dqmc.dqmc_batch_autotune(ns, b["tt_off"], arena.data_ptr(), b["dc_off"], counts.data_ptr(),
                                           bitmaps.data_ptr(), bm_off, sh, reps=3)
        tune_s = time.perf_counter() - t_tune
    table = {str(n): dqmc.dqmc_batch_get_config(int(n)) for n in sorted(set(int(x) for x in ns))}
    for _ in range(max(args.warmup, 1)):
        graph_run()
    torch.cuda.synchronize()
    K = args.steps
    sampler = ClockSampler(local) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_wall0 = time.time()
    e0.record(stream)
    for _ in range(K):
        graph_run()
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    ms = e0.elapsed_time(e1) / K
    clocks = None
    if sampler:
        time.sleep(0.3)
        sampler.stop()
        clocks = sampler.summary(t_wall0, t_wall1)
    bm_graph = bitmaps.clone()
    cnt_graph = counts.clone()

    # the same batch in one persistent launch (dqmc_batch_run_one_launch)
    def one_run():
        st = dqmc.dqmc_batch_run(ns, b["tt_off"], arena.data_ptr(), b["dc_off"], counts.data_ptr(),
                                 bitmaps.data_ptr(), bm_off, sh, one_launch=True)
        if st != 0:
            raise dqmc.DqmcError(st, "dqmc_batch_run_one_launch")

    bitmaps.zero_()
    counts.zero_()
    for _ in range(max(args.warmup, 1)):
        one_run()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        one_run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_one = e0.elapsed_time(e1) / K
    one = {"value": world * nf / (ms_one / 1e3), "unit": "functions/s", "ms_per_step": ms_one,
           "api": "dqmc_batch_run_one_launch (one persistent kernel per graph launch)",
           "results_identical": bool(torch.equal(bm_graph, bitmaps) and torch.equal(cnt_graph, counts))}
    if not one["results_identical"]:
        raise SystemExit("one-launch and graph results differ")

    if args.no_one_by_one:
        return report_batched(args, rank, world, b, nf, ns, total, ms, clocks, None, None, True, tune_s, tune_ms,
                              table, None, emit, one)

    # one launch sequence per function (dqmc_primes_dev), same buffers
    work_bytes = max(dqmc.dqmc_workspace_bytes(int(n)) for n in set(ns.tolist()))
    work = torch.empty(work_bytes, dtype=torch.uint8, device=dev)
    bitmaps.zero_()
    counts.zero_()
    nmax = np.iinfo(np.uint64).max
    a0, b0, c0, w0 = arena.data_ptr(), bitmaps.data_ptr(), counts.data_ptr(), work.data_ptr()
    calls = [(int(ns[f]), a0 + int(b["tt_off"][f]),
              None if int(b["dc_off"][f]) == nmax else a0 + int(b["dc_off"][f]),
              b0 + int(bm_off[f]), c0 + 8 * f) for f in range(nf)]

    def one_by_one():
        for n, on, dc, bm, cp in calls:
            st = L.dqmc_primes_dev(n, on, dc, bm, cp, w0, work_bytes, sh)
            if st != 0:
                raise dqmc.DqmcError(st, "dqmc_primes_dev")

    one_by_one()
    torch.cuda.synchronize()
    e0.record(stream)
    one_by_one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1)
    same = bool(torch.equal(bm_graph, bitmaps) and torch.equal(cnt_graph, counts))
    if not same:
        raise SystemExit("batched and one-by-one results differ")

    # end to end: truth tables in from pinned host memory, counts out
    e2e_s = None
    if not args.no_e2e:
        counts_h = torch.empty(nf, dtype=torch.int64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            arena.copy_(arena_h, non_blocking=True)
            graph_run()
            counts_h.copy_(counts, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / K
    return report_batched(args, rank, world, b, nf, ns, total, ms, clocks, ms_single, same, False, tune_s, tune_ms,
                          table, e2e_s, emit, one)


def report_batched(args, rank, world, b, nf, ns, total, ms, clocks, ms_single, same, skipped, tune_s, tune_ms,
                   table, e2e_s, emit=True, one=None):
    K = args.steps
    cubes = int(sum(3 ** int(n) for n in ns))
    value = world * nf / (ms / 1e3)
    result = {
        "metric": f"functions/s (batched: {nf} functions, " + (
            "n uniform in 4..14)" if args.batch_n is None else f"all n = {args.batch_n})"), "value": value,
        "unit": "functions/s", "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32 bitwise",
        "data": "synthetic",
        "config": {"workload": "batched: n = 4 + u mod 11, ON density U[0.3, 0.9], 10% with a Bernoulli(0.05) "
                               "don't-care set, seed 1+rank; step = one CUDA-graph launch of dqmc_batch_run "
                               "(bitmaps + counts of every function), tables resident in HBM",
                   "functions": nf, "cubes": cubes, "bitmap_bytes": total,
                   "l2": "no flush: the bitmaps (%.1f GB) exceed the 129 MB L2" % (total / 1e9),
                   "parallelism": f"replicas x{world}"},
        "cubes_per_s": world * cubes / (ms / 1e3),
        "one_launch_per_function": None if skipped else {
            "value": nf / (ms_single / 1e3), "unit": "functions/s", "ms_per_step": ms_single,
            "api": "dqmc_primes_dev, one call per function"},
        "speedup_vs_one_launch_per_function": None if skipped else ms_single / ms,
        "results_identical": same,
        "one_persistent_launch": one,
        "launch_table": {"autotuned": not args.no_autotune, "seconds": tune_s,
                         "best_ms_per_n": tune_ms, "config_per_n": table},
        "e2e": None if e2e_s is None else {
            "value": world * nf / e2e_s, "unit": "functions/s", "h2d_bytes_per_step": int(b["arena"].size),
            "d2h_bytes_per_step": 8 * nf},
        "clocks": clocks,
        "gpu_launches": K * launches_per_graph(ns, table),
    }
    if rank == 0 and emit:
        print(json.dumps(result), flush=True)
    return result


def launches_per_graph(ns, table):
    """Kernels one dqmc_batch_run graph launches: one per n on the shared-memory
    path and for the one-tile kernel, one per pass on the streaming path."""
    from paper_2302_10083_gb300 import dqmc
    k = 0
    for n in sorted(set(int(x) for x in ns)):
        cfg = table[str(n)]
        k += 1 if (cfg["path"] == dqmc.DQMC_BATCH_PATH_SMEM or n <= 12) else dqmc.dqmc_plan_passes(n)
    return k


def run_serving(args, rank, world, local, rates=None, emit=True):
    """Serving workload (continuous batching against one job at a time) at
    the given arrival rates; returns the result line (printed by rank 0 when
    emit)."""
    import numpy as np
    import torch

    from paper_2302_10083_gb300 import dqmc, synth

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dqmc.lib()
    rates = rates or [1e2, 1e3, 1e4, 1e5]
    m_max = args.serve_jobs
    req = synth.serving_requests(m_max, 1 + rank, rate=1.0)   # n, density, seed per job (times rescaled below)
    ns = req["n"].astype(np.uint32)
    tts = [synth.random_function(int(ns[j]), int(req["seed"][j]) & 0x7FFFFFFF, float(req["density"][j]))[0]
           for j in range(m_max)]
    budget = 64 << 30
    per_rate = []
    for lam in rates:
        m = max(1, min(m_max, int(lam * args.serve_seconds)))
        t_arr = synth.serving_requests(m, 1 + rank, rate=lam)["t_arrive"]
        t_arr = t_arr - t_arr[0]
        res = {}
        for mode, name in ((dqmc.DQMC_SERVER_CONCURRENT, "continuous"), (dqmc.DQMC_SERVER_SERIAL, "one_by_one")):
            with dqmc.Server(budget, streams=8, mode=mode) as srv:
                counts, lat, span = srv.replay(t_arr, ns[:m], tts[:m])
                st = srv.stats()
            res[name] = {"jobs_per_s": m / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                         "p99_ms": 1e3 * float(np.percentile(lat, 99)), "span_s": span,
                         "batched_launches": st["batches"], "jobs_in_batches": st["batched_jobs"],
                         "peak_running": st["peak_running"], "peak_device_bytes": st["peak_bytes"],
                         "counts": counts}
        same = bool(np.array_equal(res["continuous"].pop("counts"), res["one_by_one"].pop("counts")))
        if not same:
            raise SystemExit(f"rate {lam}: served counts differ from one-by-one")
        per_rate.append({"rate_jobs_per_s": lam, "jobs": m, **res,
                         "p99_speedup": res["one_by_one"]["p99_ms"] / res["continuous"]["p99_ms"],
                         "throughput_speedup": res["continuous"]["jobs_per_s"] / res["one_by_one"]["jobs_per_s"],
                         "counts_identical": same})
    # small jobs only (n log-uniform in 6..12), arriving faster than one job
    # at a time can serve them: the throughput of continuous batching
    m_small = 4 * m_max
    reqs = synth.serving_requests(m_small, 101 + rank, rate=1e6, n_lo=6, n_hi=12)
    ns_s = reqs["n"].astype(np.uint32)
    tts_s = [synth.random_function(int(ns_s[j]), int(reqs["seed"][j]) & 0x7FFFFFFF, float(reqs["density"][j]))[0]
             for j in range(m_small)]
    t_s = reqs["t_arrive"] - reqs["t_arrive"][0]
    small = {"rate_jobs_per_s": 1e6, "jobs": m_small, "n": "6..12"}
    cnt_s = {}
    for mode, name in ((dqmc.DQMC_SERVER_CONCURRENT, "continuous"), (dqmc.DQMC_SERVER_SERIAL, "one_by_one")):
        with dqmc.Server(budget, streams=8, mode=mode) as srv:
            counts, lat, span = srv.replay(t_s, ns_s, tts_s)
            st = srv.stats()
        cnt_s[name] = counts
        small[name] = {"jobs_per_s": m_small / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                       "p99_ms": 1e3 * float(np.percentile(lat, 99)), "span_s": span,
                       "batched_launches": st["batches"], "jobs_in_batches": st["batched_jobs"]}
    small["counts_identical"] = bool(np.array_equal(cnt_s["continuous"], cnt_s["one_by_one"]))
    if not small["counts_identical"]:
        raise SystemExit("small-job serving: counts differ from one-by-one")
    small["throughput_speedup"] = small["continuous"]["jobs_per_s"] / small["one_by_one"]["jobs_per_s"]
    top = per_rate[-1]
    result = {
        "metric": "served jobs/s at 1e5 arrivals/s (Poisson, n log-uniform 6..22), p50/p99 latency per rate",
        "value": top["continuous"]["jobs_per_s"], "unit": "jobs/s", "n_gpus": world, "steps": len(rates),
        "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 bitwise", "data": "synthetic",
        "config": {"workload": "serving: Poisson arrivals, n = floor(exp(U(ln 6, ln 23))) clipped to 6..22, "
                               "ON density U[0.2, 0.95], seed 1+rank; truth tables from host memory, "
                               "counts back to host, bitmaps device-resident until the job is done",
                   "budget_bytes": budget, "streams": 8, "parallelism": f"replicas x{world}"},
        "per_rate": per_rate,
        "small_jobs": small,
    }
    if rank == 0 and emit:
        print(json.dumps(result), flush=True)
    return result


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched":
        run_batched(args, rank, world, local)
        return 0
    if args.workload == "serving":
        run_serving(args, rank, world, local)
        return 0
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
