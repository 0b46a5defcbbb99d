#!/usr/bin/env python
"""Benchmark of the deterministic Ising max-cut annealer on GB300.

One *step* is one whole anneal of the workload: random initial spins, the full
sweep schedule (every colour class of every sweep: field gather, update, random
flip), then the energy/cut reduction. The default workload is the 1024 x 1024
torus with +-1 weights, 2000 sweeps, flip probability linear 0.1 -> 0.

Prints one JSON line (rank 0). ``value`` is spin-updates/s over all ranks with
the graph resident in HBM; ``e2e`` is the same metric through the public C ABI
starting from host edge lists (graph build and upload, anneal, cut and spins
back to host inside the timed region). ``--impl reference`` times the CPU
oracle on the host cores instead.

Multi-GPU: the path does not shard (replicas only); each rank anneals its own
replica (seed offset by rank) and ``value`` sums over ranks.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="torus1024",
                    choices=["torus1024", "zipf1m", "er800", "batched"])
    ap.add_argument("--engine", default="auto", choices=["auto", "phase", "persistent", "dataflow"])
    ap.add_argument("--mode", default="det", choices=["det", "racy"],
                    help="deterministic colour phases (bit-exact) or the racy pass")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweeps", type=int, default=None,
                    help="override the workload's schedule length (profiling runs only)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def algorithmic_bytes_per_sweep(n: int, nnz: int, entry_bytes: int) -> int:
    """Compulsory traffic of one sweep in the library's layout: every CSR entry
    streamed once (4 bytes when column and int8 weight are packed into one
    word, else 8), the int32 row offsets once, and every spin read and written
    once (int8)."""
    return nnz * entry_bytes + 4 * (n + 1) + 2 * n


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel, from ncu captures of short anneals of the same workload with the L2
# cold at launch. A launch of T sweeps moves fixed + per_sweep * T bytes; the
# per-sweep slope comes from two captures of different length (20 and 60
# sweeps) where there are two, else from one capture scaled in proportion to
# the sweeps. The entry holds only while the kernel sources hash to `sources`:
# once they change the counters are stale and traffic is reported as null.
NCU_TRAFFIC = {
    "torus1024": {"fixed": 22.3809e6, "per_sweep": 0.0, "kernel": "persistent_kernel",
                  "files": ("sweep.cuh", "anneal.cu", "philox.cuh"),
                  "sources": "aace815c91543ed2",
                  "how": "ncu 20- and 60-sweep captures: 22.383 MB and 22.379 MB, so the "
                         "working set is read once and then stays in L2"},
    "batched": {"fixed": 0.0, "per_sweep": 2.94971e9 / 20, "kernel": "batch_anneal_kernel",
                "files": ("batch.cu", "philox.cuh"),
                "sources": "b9cc8929057fad4f",
                "how": "ncu 20-sweep capture (2.950 GB) scaled in proportion to sweeps"},
}


def kernel_traffic(workload: str, sweeps: int):
    """Per-launch DRAM bytes of the dominant kernel, or None when no capture
    matches the current kernel sources."""
    import hashlib
    e = NCU_TRAFFIC.get(workload)
    if e is None:
        return None
    h = hashlib.sha256()
    for f in e["files"]:
        with open(os.path.join(ROOT, "paper_1807_10750_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != e["sources"]:
        return None
    return e["fixed"] + e["per_sweep"] * sweeps


def replica_seed(seed: int, rank: int) -> int:
    """Each rank anneals its own replica: the Philox seed is offset by rank."""
    return seed + 7919 * rank


def max_over_ranks(x: float, world: int, dist, device) -> float:
    """The slowest rank's time (the job's wall time); a no-op at world 1."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank processes the same number of units
    (weak scaling), divided by the max-over-ranks time."""
    return units_per_rank * world / seconds


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def build_workload(name, sweeps=None):
    import synth
    g, sch = synth.workload(name)
    if sweeps is not None:
        sch = dict(sch, sweeps=sweeps)
    return g, sch


def run_reference(args, world, rank):
    """The oracle as it stands, on the host cores, each step a bounded sample
    (a run of consecutive sweeps of the same schedule on the same graph)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    g, sch = build_workload(args.workload)
    T = sch["sweeps"]
    s = oracle.init_spins(g.n, sch["seed"])
    # size the per-step sample so that the whole run stays within a few minutes
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    sweeps = int(max(2, min(T, budget / oracle_sweep_cost(g, sch))))
    times = []
    t = 0
    for k in range(args.warmup + args.steps):
        if t + sweeps > T:
            t = 0
        t0 = time.perf_counter()
        s = oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=sch["seed"], p0=sch["p0"], T=T,
                          t_begin=t, sweeps=sweeps)
        dt = time.perf_counter() - t0
        t += sweeps
        if k >= args.warmup:
            times.append(dt)
    value = g.n * sweeps * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": "spin_updates_per_s", "value": value,
        "unit": "spin-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "n": g.n, "m": g.m, "sweeps_total": T,
                   "p0": sch["p0"]},
        "cpu_baseline": {"value": value, "unit": "spin-updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{sweeps} consecutive sweeps of the {T}-sweep schedule per "
                                   f"step, full graph, one oracle_anneal call (incl. its "
                                   f"adjacency rebuild) per step, single thread"},
        "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def oracle_sweep_cost(g, sch):
    """Seconds per sweep of the oracle on this graph, without the fixed cost
    of its adjacency build: two calls of different length, differenced."""
    import oracle
    oracle.build()
    T = sch["sweeps"]
    s = oracle.init_spins(g.n, sch["seed"])
    cost = []
    for k in (1, 5):
        t0 = time.perf_counter()
        oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=sch["seed"], p0=sch["p0"], T=T, sweeps=k)
        cost.append(time.perf_counter() - t0)
    return max((cost[1] - cost[0]) / 4, 1e-6)


def cpu_baseline(g, sch, target_s: float):
    import oracle
    T = sch["sweeps"]
    s = oracle.init_spins(g.n, sch["seed"])
    sweeps = int(max(2, min(T, target_s / oracle_sweep_cost(g, sch))))
    t0 = time.perf_counter()
    oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=sch["seed"], p0=sch["p0"], T=T, sweeps=sweeps)
    dt = time.perf_counter() - t0
    return {"value": g.n * sweeps / dt, "unit": "spin-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"sweeps 0..{sweeps - 1} of the {T}-sweep schedule on the full graph "
                      f"({dt:.1f} s, single thread, one oracle_anneal call incl. adjacency build)"}


def run_batched(args, world, rank, P, torch, dist):
    """The batched workload: 1024 instances x 8 replicas, 1000 sweeps, one
    persistent kernel (captured in a CUDA graph) per step."""
    import synth
    gs, sch = synth.batched_workload()
    if args.sweeps is not None:
        sch = dict(sch, sweeps=args.sweeps)
    T, p0, R = sch["sweeps"], sch["p0"], sch["replicas"]
    seed = replica_seed(sch["seed"], rank)
    stream = torch.cuda.Stream()
    arrays = [(g.n, g.src, g.dst, g.w) for g in gs]
    b = P.ising_batch_create(arrays, replicas=R, stream=stream)
    block = P.ising_batch_autotune(b, probe_sweeps=20)
    nvert = sum(g.n for g in gs)
    nnz = 2 * sum(g.m for g in gs)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def step(k):
        P.ising_batch_init_random(b, seed + k)
        ev[0].record(stream)
        P.ising_batch_anneal(b, p0=p0, t_total=T, seed=seed + k, stream=stream)
        ev[1].record(stream)
        return P.ising_batch_cuts(b)

    for k in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        step(k)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    anneal_ms, best = [], []
    launches0 = P.ising_batch_info(b)["launches"]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            starts[k].record(stream)
            cuts = step(args.warmup + k)
            ends[k].record(stream)
            torch.cuda.synchronize()
            anneal_ms.append(ev[0].elapsed_time(ev[1]))
            best.append(float(cuts.max(axis=1).sum()))
    launches = P.ising_batch_info(b)["launches"] - launches0
    total_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    total_ms = max_over_ranks(total_ms, world, dist, "cuda")
    value = job_throughput(nvert * R * T * args.steps, world, total_ms / 1e3)
    # per sweep every instance's packed CSR words, row offsets and vertex ids
    # are read once; spins live in shared memory
    B = nnz * 4 + 4 * (nvert + len(gs)) + 4 * nvert
    sweep_s = (sum(anneal_ms) / len(anneal_ms)) / 1e3 / T
    achieved = B / sweep_s / 1e9
    peak, peak_kind = measured_peaks()
    e2e = None
    if args.e2e_steps > 0:
        e2e_t = []
        for k in range(args.e2e_steps + 1):
            t0 = time.perf_counter()
            with P.ising_batch_create(arrays, replicas=R, stream=stream) as b2:
                P.ising_batch_set_block(b2, block)
                P.ising_batch_init_random(b2, seed + k)
                P.ising_batch_anneal(b2, p0=p0, t_total=T, seed=seed + k, stream=stream)
                P.ising_batch_cuts(b2)
            if k > 0:
                e2e_t.append(time.perf_counter() - t0)
        e2e_total = sum(e2e_t)
        e2e_total = max_over_ranks(e2e_total, world, dist, "cuda")
        e2e = {"value": nvert * R * T * len(e2e_t) * world / e2e_total, "unit": "spin-updates/s",
               "h2d_bytes_per_step": int(12 * sum(g.m for g in gs) + 4 * len(gs) + 8 * len(gs)),
               "d2h_bytes_per_step": int(8 * len(gs) * R),
               "ms_per_step": 1e3 * e2e_total / len(e2e_t)}
    if rank != 0:
        return
    line = {
        "metric": "spin_updates_per_s", "value": value, "unit": "spin-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
        "data": "synthetic",
        "config": {"workload": "batched", "instances": len(gs), "vertices": nvert,
                   "edges": nnz // 2, "replicas": R, "sweeps": T, "p0": p0, "block": block,
                   "parallelism": f"replicas{world}",
                   "l2": "512 MiB buffer zeroed between timed steps (outside the events)"},
        "sweeps_per_s": T * args.steps * world / (total_ms / 1e3),
        "best_cut_sum_mean": float(np.mean(best)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": kernel_traffic("batched", T),
                     "peak_kind": peak_kind, "bytes_per_sweep": B, "bytes_per_launch": B * T,
                     "kernel": "batch_anneal_kernel (one launch per step)"},
        "cpu_baseline": None, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import torch.distributed as dist

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_1807_10750_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        dist.barrier()
    import paper_1807_10750_gb300 as P

    if args.workload == "batched":
        run_batched(args, world, rank, P, torch, dist)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    g, sch = build_workload(args.workload, args.sweeps)
    T, p0, seed = sch["sweeps"], sch["p0"], replica_seed(sch["seed"], rank)
    stream = torch.cuda.Stream()
    engine = {"auto": P.ISING_ENGINE_AUTO, "phase": P.ISING_ENGINE_PHASE,
              "persistent": P.ISING_ENGINE_PERSISTENT,
              "dataflow": P.ISING_ENGINE_DATAFLOW}[args.engine]

    h = P.ising_create(g.n, g.src, g.dst, g.w, stream=stream)
    P.ising_set_engine(h, engine)
    mode = P.ISING_MODE_RACY if args.mode == "racy" else P.ISING_MODE_DET
    # AUTO resolves to the persistent engine on devices with cooperative launch
    engine_name = "persistent" if args.engine == "auto" else args.engine
    colours = P.ising_num_colours(h)
    m = P.ising_num_edges(h)
    nnz = 2 * m
    w_bytes = 1 if np.abs(g.w).max(initial=0) <= 127 else 4
    # the library packs (column, int8 weight) into one int32 when it can
    entry_bytes = 4 if (w_bytes == 1 and g.n < (1 << 24) - 1) else 8
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def step(k):
        P.ising_init_random(h, seed + k)
        ev[0].record(stream)
        P.ising_anneal(h, p0=p0, t_total=T, seed=seed + k, stream=stream, mode=mode)
        ev[1].record(stream)
        return P.ising_cut(h)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for k in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        step(k)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    anneal_ms = []
    cuts = []
    launches0 = P.ising_launch_count(h)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clocks:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()            # L2 flush between steps (outside the timed events)
            starts[k].record(stream)
            cuts.append(step(args.warmup + k))
            ends[k].record(stream)
            torch.cuda.synchronize()
            anneal_ms.append(ev[0].elapsed_time(ev[1]))
    torch.cuda.synchronize()
    launches = P.ising_launch_count(h) - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, world, dist, "cuda")
    if world > 1:
        dist.barrier()
    value = job_throughput(g.n * T * args.steps, world, total_ms / 1e3)

    # roofline of the sweep kernels: algorithmic bytes per sweep / time per sweep
    B = algorithmic_bytes_per_sweep(g.n, nnz, entry_bytes)
    sweep_s = (sum(anneal_ms) / len(anneal_ms)) / 1e3 / T
    achieved = B / sweep_s / 1e9
    peak, peak_kind = measured_peaks()

    # end to end through the C ABI from pinned host edge lists
    e2e = None
    if args.e2e_steps > 0:
        src_p = torch.from_numpy(g.src).pin_memory().numpy()
        dst_p = torch.from_numpy(g.dst).pin_memory().numpy()
        w_p = torch.from_numpy(g.w).pin_memory().numpy()
        spins_out = torch.empty(g.n, dtype=torch.int8).pin_memory().numpy()
        torch.cuda.synchronize()
        e2e_t = []
        for k in range(args.e2e_steps + 1):
            t0 = time.perf_counter()
            with P.ising_create(g.n, src_p, dst_p, w_p, stream=stream) as h2:
                P.ising_set_engine(h2, engine)
                P.ising_init_random(h2, seed + k)
                P.ising_anneal(h2, p0=p0, t_total=T, seed=seed + k, stream=stream, mode=mode)
                P.ising_cut(h2)
                P.ising_get_spins(h2, spins_out)
            dt = time.perf_counter() - t0
            if k > 0:
                e2e_t.append(dt)
        e2e_total = sum(e2e_t)
        e2e_total = max_over_ranks(e2e_total, world, dist, "cuda")
        e2e = {"value": g.n * T * len(e2e_t) * world / e2e_total, "unit": "spin-updates/s",
               "h2d_bytes_per_step": int(3 * 4 * g.m), "d2h_bytes_per_step": int(g.n + 8),
               "ms_per_step": 1e3 * e2e_total / len(e2e_t)}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g, sch, args.cpu_seconds)

    line = {
        "metric": "spin_updates_per_s",
        "value": value,
        "unit": "spin-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int8",
        "data": "synthetic",
        "config": {
            "workload": args.workload, "n": g.n, "m": m, "colours": colours,
            "sweeps": T, "p0": p0, "schedule": "linear",
            "mode": "racy" if args.mode == "racy" else "deterministic",
            "engine": args.engine, "weights": "int8" if w_bytes == 1 else "int32",
            "csr_entry_bytes": entry_bytes,
            "replicas_per_gpu": 1, "parallelism": f"replicas{world}",
            "l2": "512 MiB buffer zeroed between timed steps (outside the events)",
        },
        "sweeps_per_s": T * args.steps * world / (total_ms / 1e3),
        "algorithmic_gbs": achieved,
        "final_cut_mean": float(np.mean(cuts)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (kernel_traffic(args.workload, T)
                                 if engine_name == "persistent" and args.mode == "det"
                                 else None),
                     "peak_kind": peak_kind, "bytes_per_sweep": B, "bytes_per_launch": B * T,
                     "kernel": f"{engine_name} sweep kernel(s) of one anneal call"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    P.ising_destroy(h)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
