#!/usr/bin/env python
"""Benchmark of the deterministic Ising max-cut annealer on GB300.

One *step* is one whole anneal of the workload: random initial spins, the full
sweep schedule (every colour class of every sweep: field gather, update, random
flip), then the energy/cut reduction. The default workload is the 2^20-vertex
power-law graph (erased configuration model, degrees ~ d^-2.1 on [4, 10000],
weights uniform in [-8, 8] without 0), 2000 sweeps, flip probability linear
0.1 -> 0. ``--workload all`` prints one line for every workload (the 800-vertex
random graph, the 1024 x 1024 torus, the power-law graph, the batched set and
the learned warm start), each from its own process.

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
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: per workload, a timed region of several seconds)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=None,
                    choices=["torus1024", "zipf1m", "er800", "batched", "warmstart", "gnn", "region",
                             "all"])
    ap.add_argument("--engine", default="auto",
                    choices=["auto", "phase", "persistent", "dataflow", "persistent_grid", "itemflow",
                             "halo", "hub"])
    ap.add_argument("--halo-sweeps", type=int, default=0,
                    help="sweeps per exchange of the halo engine (0: automatic)")
    ap.add_argument("--mode", default="det", choices=["det", "racy"],
                    help="deterministic colour phases (bit-exact) or the racy pass")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweeps", type=int, default=None,
                    help="override the workload's schedule length (profiling runs only)")
    ap.add_argument("--gnn-dense", choices=["mma_sync", "tcgen05"], default="mma_sync",
                    help="gnn: the forward layers' product (ising_gnn_set_dense_path)")
    ap.add_argument("--train-graphs", type=int, default=2048,
                    help="warmstart: generated training graphs (1k-100k vertices)")
    ap.add_argument("--train-batch", type=int, default=64,
                    help="warmstart: training graphs per batch (one Adam step each)")
    ap.add_argument("--train-steps", type=int, default=1500, help="warmstart: Adam steps")
    ap.add_argument("--test-graphs", type=int, default=152,
                    help="warmstart: held-out 100k-vertex power-law graphs")
    ap.add_argument("--long-sweeps", type=int, default=20000,
                    help="warmstart: sweeps of the long run that sets each graph's best cut")
    ap.add_argument("--plain-sweeps", type=lambda t: [int(x) for x in t.split(",")],
                    default=[100, 200, 400, 800, 1600, 3200, 6400],
                    help="warmstart: the plain anneal lengths timed")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def algorithmic_bytes_per_sweep(n: int, nnz: int, entry_bytes: int) -> int:
    """Compulsory traffic of one sweep: every directed CSR entry streamed once
    (an int32 column index plus the weight: 4 + 1 bytes for int8 weights,
    4 + 4 for int32), the int32 row offsets once, and every int8 spin read and
    written once. `entry_bytes` is the column plus weight size."""
    return nnz * entry_bytes + 4 * (n + 1) + 2 * n


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel, from ncu captures of short anneals of the same workload with the L2
# cold at launch. A launch of T sweeps moves fixed + per_sweep * T bytes; the
# per-sweep slope comes from two captures of different length (20 and 60
# sweeps) where there are two, else from one capture scaled in proportion to
# the sweeps. The entry holds only while the kernel sources hash to `sources`:
# once they change the counters are stale and traffic is reported as null.
NCU_TRAFFIC = {
    "zipf1m": {"fixed": 99.3e6, "per_sweep": 11.61e6, "kernel": "hub_kernel", "engine": "hub",
               "files": ('hub.cuh', 'sweep.cuh', 'philox.cuh', 'anneal.cu'),
               "sources": "263febaf28510827",
               "how": "ncu 4- and 12-sweep captures: 145.73 MB and 238.62 MB (read + write); the "
                      "CSR is read from DRAM once and then mostly served from L2"},
    "torus1024": {"fixed": 31.79e6, "per_sweep": 4.03e3, "kernel": "halo_kernel",
                  "engine": "halo",
                  "files": ('halo.cuh', 'halo_plan.cpp', 'host_graph.h', 'philox.cuh', 'sweep.cuh'),
                  "sources": "6bf5d71760ec383b",
                  "how": "ncu 20- and 40-sweep captures: 31.870 MB and 31.951 MB, so the "
                         "working set is read once and then stays in shared memory and L2"},
    "batched": {"fixed": 0.2126e9, "per_sweep": 0.2083e9, "kernel": "batch_anneal_kernel",
                "files": ('batch.cu', 'philox.cuh'),
                "sources": "cb30dcc0eb10999b",
                "how": "ncu 20- and 60-sweep captures: 4.379 GB and 12.710 GB"},
}


def kernel_traffic(workload: str, sweeps: int, engine: str = ""):
    """Per-launch DRAM bytes of the dominant kernel, or None when no capture
    matches the workload, the engine that ran, or the current kernel sources."""
    import hashlib
    e = NCU_TRAFFIC.get(workload)
    if e is None or (engine and e.get("engine", engine) != engine):
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
    budget = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    per_sweep, setup = oracle_sweep_cost(g, sch)
    sweeps = int(max(2, min(T, budget / per_sweep)))
    times = []
    t = 0
    for k in range(args.warmup + args.steps):
        if t + sweeps > T:
            t = 0
        t0 = time.perf_counter()
        s = oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=sch["seed"], p0=sch["p0"], T=T,
                          t_begin=t, sweeps=sweeps)
        # the oracle rebuilds its adjacency and colouring on every call: that
        # fixed cost (a zero-sweep call, measured) is not sweep work
        dt = max(time.perf_counter() - t0 - setup, 1e-9)
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
                                   f"step, full graph, one oracle_anneal call per step minus "
                                   f"its measured {setup:.2f} s adjacency and colouring rebuild, "
                                   f"single thread"},
        "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def oracle_sweep_cost(g, sch):
    """(seconds per sweep, seconds of fixed setup) of the oracle on this graph.
    Every oracle call rebuilds its adjacency and colouring; a zero-sweep call
    measures that setup, and a short call less the setup gives the per-sweep
    cost (never below a tenth of the short call's time per sweep)."""
    import oracle
    oracle.build()
    T = sch["sweeps"]
    s = oracle.init_spins(g.n, sch["seed"])
    t0 = time.perf_counter()
    oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=sch["seed"], p0=sch["p0"], T=T, sweeps=0)
    setup = time.perf_counter() - t0
    k = min(8, T)
    t0 = time.perf_counter()
    oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=sch["seed"], p0=sch["p0"], T=T, sweeps=k)
    call = time.perf_counter() - t0
    return max((call - setup) / k, 0.1 * call / k, 1e-6), setup


def cpu_baseline(g, sch, target_s: float):
    import oracle
    T = sch["sweeps"]
    s = oracle.init_spins(g.n, sch["seed"])
    per_sweep, setup = oracle_sweep_cost(g, sch)
    sweeps = int(max(2, min(T, target_s / per_sweep)))
    t0 = time.perf_counter()
    oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=sch["seed"], p0=sch["p0"], T=T, sweeps=sweeps)
    dt = max(time.perf_counter() - t0 - setup, 1e-9)
    return {"value": g.n * sweeps / dt, "unit": "spin-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"sweeps 0..{sweeps - 1} of the {T}-sweep schedule on the full graph "
                      f"({dt:.1f} s of sweeps, single thread: one oracle_anneal call less its "
                      f"measured {setup:.2f} s adjacency and colouring rebuild)"}


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
    tuning = P.ising_batch_tuning(b)
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
                P.ising_batch_set_tuning(b2, tuning["block"], tuning["row_split"], tuning["tail"])
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
                   "tuning": {"block": tuning["block"], "row_split": tuning["row_split"],
                              "tail": tuning["tail"],
                              "probe_ms_20_sweeps": [round(x, 3) for x in tuning["probe_ms"]],
                              "probe_order": "6 * block(128,256,512) + 2 * row_split(1,2,4) + tail(0,32)"},
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


def _warmstart_graph(spec):
    """Build one generated graph (a process-pool task)."""
    import synth
    g = synth.graph_from_spec(spec)
    return (g.n, g.src, g.dst, g.w)


def run_warmstart(args, world, rank, P, torch, dist):
    """The learned warm start against the plain annealer, batched, on
    held-out graphs.

    Untimed set-up. Training data from the annealer itself: generated graphs
    (power-law and Erdos-Renyi alternately, 1k-100k vertices) in batches of
    `--train-batch` instances; per batch, input = the spins after a 100-sweep
    anneal, label = the spins after a further 200-sweep anneal at p0 = 0.01.
    The network trains on the GPU, one Adam step per batch of instances
    (ising_gnn_batch_train_step). The held-out power-law graphs form one
    batch of 8 replicas; the long-run best cut of each graph is the best of
    its 8 replicas after `--long-sweeps` sweeps.

    Timed (CUDA events on the batch's stream, from random spins): plain
    batch anneals of T sweeps, and the learned form -- a short anneal, then
    rounds of (network warm start of every replica + 10 greedy sweeps).
    Reported: for each form the least time at which every held-out graph has
    a replica at 99 % of its best cut."""
    import multiprocessing as mp
    import synth
    train_specs, test_specs, spec = synth.warmstart_specs(
        synth.WARMSTART_BATCHED, train_count=args.train_graphs, test_count=args.test_graphs)
    per = max(1, args.train_batch)
    stream = torch.cuda.Stream()
    seed0 = 1000 + 7919 * rank
    t_setup = time.perf_counter()
    pool = mp.get_context("spawn").Pool(processes=max(1, min(16, os.cpu_count() or 1)))
    chunks = [train_specs[i:i + per] for i in range(0, len(train_specs), per)]
    pending = pool.map_async(_warmstart_graph, chunks[0]) if chunks else None
    gen_s = label_s = 0.0
    train_vertices = 0
    batches = []
    for ci in range(len(chunks)):
        tg = time.perf_counter()
        graphs = pending.get()
        pending = pool.map_async(_warmstart_graph, chunks[ci + 1]) if ci + 1 < len(chunks) else None
        gen_s += time.perf_counter() - tg
        tl = time.perf_counter()
        b = P.ising_batch_create(graphs, replicas=1, stream=stream)
        sd = seed0 + 17 * ci
        P.ising_batch_init_random(b, sd)
        P.ising_batch_anneal(b, p0=0.1, t_total=100, seed=sd, stream=stream)
        snap = [P.ising_batch_get_spins(b, k, 0) for k in range(len(graphs))]
        P.ising_batch_anneal(b, p0=0.01, t_total=200, seed=sd + 5000, stream=stream)
        lab = np.concatenate([P.ising_batch_get_spins(b, k, 0) for k in range(len(graphs))])
        for k, sp in enumerate(snap):
            P.ising_batch_set_spins(b, k, 0, sp)
        batches.append((b, torch.from_numpy(lab).to("cuda")))
        train_vertices += lab.size
        label_s += time.perf_counter() - tl
        del graphs, snap
    tg = time.perf_counter()
    test_graphs = pool.map(_warmstart_graph, test_specs)
    gen_s += time.perf_counter() - tg
    pool.close()
    pool.join()

    net = P.ising_gnn_create(synth.gnn_init_params(spec["gen_seed"]))
    steps = args.train_steps
    rng = np.random.default_rng(spec["gen_seed"])
    order = []
    losses = []
    torch.cuda.synchronize()
    t_train = time.perf_counter()
    for it in range(steps):
        if not order:
            order = list(rng.permutation(len(batches)))
        b, lab = batches[order.pop()]
        lr = 2e-3 if it < 3 * steps // 4 else 5e-4
        loss = P.ising_gnn_batch_train_step(net, b, lab, lr=lr,
                                            want_loss=(it % 250 == 0 or it == steps - 1))
        if loss is not None:
            losses.append(round(loss, 4))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t_train
    for b, _ in batches:
        b.close()
    batches = []

    tb = P.ising_batch_create(test_graphs, replicas=8, stream=stream)
    num = len(test_graphs)
    test_vertices = sum(g[0] for g in test_graphs)
    del test_graphs
    P.ising_batch_init_random(tb, 1)
    P.ising_batch_autotune(tb, 10)
    tuning = P.ising_batch_tuning(tb)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        torch.cuda.synchronize()
        ev[0].record(stream)
        fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3

    def graph_best():
        return P.ising_batch_cuts(tb).reshape(num, 8).max(axis=1)

    # long-run best of every held-out graph
    P.ising_batch_init_random(tb, 90001)
    long_s = timed(lambda: P.ising_batch_anneal(tb, p0=0.1, t_total=args.long_sweeps, seed=90001,
                                                stream=stream))
    long_best = graph_best()
    # untimed: the network's workspace and the union's row tables
    P.ising_gnn_batch_forward(net, tb, 0, torch.empty(test_vertices, dtype=torch.float32, device="cuda"))
    fwd_s = timed(lambda: P.ising_gnn_batch_forward(
        net, tb, 0, torch.empty(test_vertices, dtype=torch.float32, device="cuda")))
    plain = []
    for T in args.plain_sweeps:
        P.ising_batch_init_random(tb, 7)
        sec = timed(lambda: P.ising_batch_anneal(tb, p0=0.1, t_total=T, seed=7, stream=stream))
        plain.append({"sweeps": T, "s": sec, "cuts": graph_best()})
    learned = []
    for Ta in (25, 50, 100):
        for rounds in (1, 2, 4, 8):
            P.ising_batch_init_random(tb, 7)

            def run():
                P.ising_batch_anneal(tb, p0=0.1, t_total=Ta, seed=7, stream=stream)
                for r in range(rounds):
                    P.ising_gnn_batch_warm_start(net, tb)
                    P.ising_batch_anneal(tb, p0=0.0, t_total=10, seed=11 + r, stream=stream)
            sec = timed(run)
            learned.append({"prefix": Ta, "rounds": rounds, "s": sec, "cuts": graph_best()})
    tb.close()
    net.close()
    best = np.maximum.reduce([long_best] + [c["cuts"] for c in plain + learned])

    def summarise(curve, ref):
        out = []
        for c in curve:
            ratio = c["cuts"] / np.maximum(ref, 1)
            d = {k: v for k, v in c.items() if k != "cuts"}
            d.update({"min_ratio": float(ratio.min()), "mean_ratio": float(ratio.mean()),
                      "graphs_at_99": int(np.sum(ratio >= 0.99))})
            out.append(d)
        return out

    def first(curve):
        ok = [c["s"] for c in curve if c["graphs_at_99"] == num]
        return min(ok) if ok else None
    plain_c, learned_c = summarise(plain, best), summarise(learned, best)
    plain_lr, learned_lr = summarise(plain, long_best), summarise(learned, long_best)
    if rank != 0:
        return
    value, plain_value = first(learned_c), first(plain_c)
    # where the plain annealer never got there, its longest timed run bounds
    # its time from below
    plain_bound = plain_value if plain_value is not None else max(c["s"] for c in plain_c)
    line = {
        "metric": "time_to_cut_99pct_of_best", "value": value, "unit": "s", "n_gpus": world,
        "steps": len(plain) + len(learned), "warmup": 0, "ms_per_step": None if value is None else value * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int8+bf16",
        "data": "synthetic",
        "config": {"workload": "warmstart", "form": "batched", "train_graphs": len(train_specs),
                   "train_vertices": int(train_vertices), "train_n_range": [spec["nmin"], spec["nmax"]],
                   "train_batch": per, "train_steps": steps, "test_graphs": num, "test_n": spec["test_n"],
                   "replicas": 8, "best_of": f"max(best of 8 replicas x {args.long_sweeps} sweeps at p0 0.1, "
                                             "every timed run), per graph",
                   "reached": "every held-out graph has a replica at >= 99 % of its best cut",
                   "learned_form": "anneal(prefix sweeps, p0 0.1) + rounds x (network warm start of every "
                                   "replica + 10 greedy sweeps)",
                   "batch_tuning": tuning, "parallelism": f"replicas{world}"},
        "plain_value": plain_value,
        "plain_value_lower_bound": plain_bound,
        "speedup_vs_plain": None if value is None or plain_value is None else plain_value / value,
        "speedup_vs_plain_lower_bound": None if value is None else plain_bound / value,
        "of_long_run_best": {"learned_s": first(learned_lr), "plain_s": first(plain_lr)},
        "plain": plain_c, "learned": learned_c,
        "long_run_s": long_s, "forward_one_replica_s": fwd_s,
        "generate_s": gen_s, "label_s": label_s, "train_s": train_s,
        "setup_s": time.perf_counter() - t_setup, "train_loss": losses,
        "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": None,
    }
    print(json.dumps(line), flush=True)


def gnn_forward_bytes(n: int, nnz: int) -> int:
    """Compulsory bytes of one forward pass of the warm-start network: row
    sums (CSR word, row id, neighbour spin per entry; an int4 per row out),
    features (sums, spin in; 8 bf16 features and c out), three layers (per
    entry the CSR word, c_j and the neighbour's bf16 feature row; per row its
    row bounds, c, its own row in and its 64-wide bf16 output) and the head
    (h3 in, z out). The aggregate a never leaves the layer kernel, so it
    moves no bytes."""
    rowsum = nnz * 9 + n * 16
    feats = n * (16 + 1 + 16 + 4)
    layer8 = nnz * (8 + 16) + n * (12 + 16 + 128)
    layer64 = nnz * (8 + 128) + n * (12 + 128 + 128)
    head = n * (128 + 4)
    return rowsum + feats + layer8 + 2 * layer64 + head


def run_gnn(args, world, rank, P, torch, dist):
    """Throughput of the warm-start network's kernels on a held-out-sized
    graph (100k-vertex power-law graph, random parameters): forward passes
    and training steps (forward, backward, Adam) per second."""
    import synth
    _, test, spec = synth.warmstart_workload(train_count=0, test_count=1)
    g = test[0]
    stream = torch.cuda.Stream()
    h = P.ising_create(g.n, g.src, g.dst, g.w, stream=stream)
    P.ising_init_random(h, 1)
    net = P.ising_gnn_create(synth.gnn_init_params(1))
    P.ising_gnn_set_dense_path(net, P.ISING_GNN_DENSE_TCGEN05 if args.gnn_dense == "tcgen05"
                               else P.ISING_GNN_DENSE_MMA_SYNC)
    z = torch.empty(g.n, dtype=torch.float32, device="cuda")
    y = torch.from_numpy(np.where(np.random.default_rng(2).random(g.n) < 0.5, 1, -1).astype(np.int8)).cuda()
    nnz = 2 * P.ising_num_edges(h)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(args.warmup):
        P.ising_gnn_forward(net, h, z)
        P.ising_gnn_train_step(net, h, y, lr=0.0)
    torch.cuda.synchronize()
    fwd, trn = [], []
    l0 = P.ising_gnn_launch_count(net)
    with ClockSampler(torch.cuda.current_device()) as clocks:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[0].record(stream)
            P.ising_gnn_forward(net, h, z)
            ev[1].record(stream)
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[2].record(stream)
            P.ising_gnn_train_step(net, h, y, lr=0.0)
            ev[3].record(stream)
            torch.cuda.synchronize()
            fwd.append(ev[0].elapsed_time(ev[1]))
            trn.append(ev[2].elapsed_time(ev[3]))
    launches = P.ising_gnn_launch_count(net) - l0
    fwd_ms = statistics.median(fwd)
    trn_ms = statistics.median(trn)
    B = gnn_forward_bytes(g.n, nnz)
    achieved = B / (fwd_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    if rank != 0:
        return
    line = {
        "metric": "gnn_forward_vertices_per_s", "value": g.n / (fwd_ms / 1e3) * world,
        "unit": "vertices/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": fwd_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "gnn", "n": g.n, "nnz": nnz, "layers": 3, "hidden": 64,
                   "dense": args.gnn_dense.replace("_", "."),
                   "parallelism": f"replicas{world}",
                   "l2": "512 MiB buffer zeroed before every timed pass (outside the events)"},
        "train_step_ms": trn_ms, "train_vertices_per_s": g.n / (trn_ms / 1e3) * world,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                     "bytes_per_forward": B, "kernel": "all kernels of one forward pass"},
        "cpu_baseline": None, "e2e": None,
        "gpu_launches": int(launches), "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    h.close()
    net.close()


# Shared-memory traffic of the halo kernel per sweep: l1tex shared-memory
# wavefronts (one wavefront moves up to 128 bytes) from ncu captures, slope
# over the sweep count; valid while the kernel sources hash to `sources`.
NCU_SMEM = {
    "torus1024": {"wavefronts_per_sweep": 575_506,
                  "files": ('halo.cuh', 'halo_plan.cpp', 'host_graph.h', 'philox.cuh', 'sweep.cuh'),
                  "sources": "6bf5d71760ec383b",
                  "how": "l1tex__data_pipe_lsu_wavefronts_mem_shared.sum: 11,810,305 (20 sweeps) and "
                         "23,320,433 (40 sweeps)"},
}


def roofline_entry(args, engine_name, T, B, B_lib, achieved, peak, peak_kind, sweep_s, clk):
    """The roofline object of the dominant kernel. The grid and hub engines
    stream the CSR through L2 and HBM every sweep: bound "hbm", achieved =
    algorithmic bytes (5 bytes per directed entry with int8
    weights) over time. The halo engine reads its part of the graph from HBM
    once per launch and then works from shared memory, so its bound is the
    SMs' shared-memory bandwidth (152 SMs x 128 bytes per clock at the
    sampled SM clock); the HBM figure is kept as a labelled secondary one."""
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak,
           "traffic": (kernel_traffic(args.workload, T, engine_name) if args.mode == "det" else None),
           "peak_kind": peak_kind, "bytes_per_sweep": B, "bytes_per_launch": B * T,
           "bytes_per_sweep_library_layout": B_lib,
           "kernel": f"{engine_name} sweep kernel(s) of one anneal call"}
    if engine_name != "halo":
        return hbm
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    smem_peak = sms * 128 * mhz * 1e6 / 1e9
    e = NCU_SMEM.get(args.workload)
    smem_bytes = None
    if e is not None:
        import hashlib
        h = hashlib.sha256()
        for f in e["files"]:
            with open(os.path.join(ROOT, "paper_1807_10750_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest()[:16] == e["sources"]:
            smem_bytes = 128 * e["wavefronts_per_sweep"]
    smem_achieved = smem_bytes / sweep_s / 1e9 if smem_bytes else None
    return {"bound": "smem", "achieved": smem_achieved, "peak": smem_peak, "unit": "GB/s",
            "frac": smem_achieved / smem_peak if smem_achieved else None,
            "traffic": hbm["traffic"], "peak_kind": "nominal: SMs x 128 B/clock x sampled SM clock",
            "smem_bytes_per_sweep": smem_bytes,
            "kernel": "halo_kernel (one launch per anneal call)",
            "hbm_secondary": {k: hbm[k] for k in ("achieved", "peak", "frac", "bytes_per_sweep",
                                                   "bytes_per_launch", "peak_kind")}}


WORKLOADS_ALL = ["er800", "torus1024", "zipf1m", "batched", "warmstart", "region"]


def run_all(args):
    """One line per workload, each from its own process with the same flags."""
    if dist_env()[0] > 1:
        raise SystemExit("--workload all runs on one GPU (no torchrun)")
    rc = 0
    # the CPU oracle arm covers the single-graph workloads
    names = WORKLOADS_ALL if args.impl == "ours" else ["er800", "torus1024", "zipf1m"]
    for wl in names:
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", wl,
               "--warmup", str(args.warmup), "--impl", args.impl, "--e2e-steps", str(args.e2e_steps),
               "--cpu-seconds", str(args.cpu_seconds)]
        if args.steps is not None:
            cmd += ["--steps", str(args.steps)]
        if wl == "warmstart":  # the reduced form of the default run's secondary line
            cmd += [x for x in dict((n, e) for n, e, _ in SECONDARY)["warmstart"] if x not in ("--workload", "warmstart")]
        if args.no_cpu_baseline:
            cmd.append("--no-cpu-baseline")
        r = subprocess.run(cmd, stdout=subprocess.PIPE, text=True)
        sys.stdout.write(r.stdout)
        sys.stdout.flush()
        rc = rc or r.returncode
    raise SystemExit(rc)


def run_region(args, world, rank, P, torch, dist):
    """The paper's convergence study (Sec. V-C, Fig. 4) on the 800-vertex
    random graph: 10 seeded runs of the 1000-sweep schedule, the cut after
    every 50 sweeps, and its min / max over the runs (ising_convergence_region).
    The timed quantity is the whole region (10 runs and their checkpoints)."""
    g, sch = build_workload("er800", args.sweeps)
    T, p0 = sch["sweeps"], sch["p0"]
    every, seeds = 50, [sch["seed"] + 7919 * rank + k for k in range(10)]
    stream = torch.cuda.Stream()
    h = P.ising_create(g.n, g.src, g.dst, g.w, stream=stream)
    for _ in range(args.warmup):
        P.ising_convergence_region(h, seeds=seeds, p0=p0, t_total=T, every=every, stream=stream)
    torch.cuda.synchronize()
    times = []
    launches0 = P.ising_launch_count(h)
    with ClockSampler(torch.cuda.current_device()) as clocks:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            idx, cuts, lo, hi = P.ising_convergence_region(h, seeds=seeds, p0=p0, t_total=T,
                                                           every=every, stream=stream)
            times.append(time.perf_counter() - t0)
    launches = P.ising_launch_count(h) - launches0
    total = max_over_ranks(sum(times), world, dist, "cuda")
    if rank == 0:
        line = {
            "metric": "spin_updates_per_s", "value": g.n * T * len(seeds) * args.steps * world / total,
            "unit": "spin-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": {"workload": "region", "graph": "er800", "n": g.n, "m": P.ising_num_edges(h),
                       "sweeps": T, "p0": p0, "runs": len(seeds), "every": every,
                       "parallelism": f"replicas{world}",
                       "timing": "host wall clock around each ising_convergence_region call "
                                 "(it synchronises after every chunk)"},
            "region": {"sweep": idx.tolist(), "min_cut": lo.tolist(), "max_cut": hi.tolist(),
                       "one_run_cut": cuts[0].tolist(), "mean_final_cut": float(cuts[:, -1].mean())},
            "roofline": None, "cpu_baseline": None, "e2e": None,
            "gpu_launches": int(launches), "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    h.close()


# The lines a default run (no --workload) adds under "secondary", each from
# its own process after the headline zipf1m measurement: the batched workload
# and a reduced batched warm-start run (the full-scale run is
# --workload warmstart --train-graphs 20000 --train-batch 256 --test-graphs 152
# --long-sweeps 20000).
SECONDARY = [
    ("batched", ["--workload", "batched", "--warmup", "3", "--e2e-steps", "1"], 900),
    ("warmstart", ["--workload", "warmstart", "--train-graphs", "512", "--train-steps", "400",
                   "--test-graphs", "32", "--long-sweeps", "4000",
                   "--plain-sweeps", "100,200,400,800,1600,3200"], 1200),
]


def run_secondary():
    """Run the SECONDARY workloads, one process each; their JSON lines (or
    what went wrong)."""
    out = []
    for name, extra, limit in SECONDARY:
        cmd = [sys.executable, os.path.abspath(__file__), "--no-cpu-baseline"] + extra
        try:
            r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=limit)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            if r.returncode == 0 and lines:
                out.append(json.loads(lines[-1]))
            else:
                out.append({"workload": name, "error": f"exit {r.returncode}: {r.stderr.strip()[-300:]}"})
        except subprocess.TimeoutExpired:
            out.append({"workload": name, "error": f"did not finish within {limit} s"})
    return out


# Default timed steps per workload: each timed region covers several seconds
# (zipf1m 30 x 0.49 s, torus1024 300 x 11.6 ms, er800 200 x 17.8 ms, the
# batched workload 25 x 140 ms, the region 20 x 0.18 s).
DEFAULT_STEPS = {"zipf1m": 30, "torus1024": 300, "er800": 200, "batched": 25, "region": 20, "gnn": 20}


def main():
    args = parse_args()
    secondary = args.workload is None and args.impl == "ours" and args.sweeps is None
    if args.workload is None:
        args.workload = "zipf1m"
    if args.steps is None and args.workload != "all":
        args.steps = DEFAULT_STEPS.get(args.workload, 30)
    if args.workload == "all":
        run_all(args)
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

    if args.workload == "gnn":
        run_gnn(args, world, rank, P, torch, dist)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    if args.workload == "warmstart":
        run_warmstart(args, world, rank, P, torch, dist)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    if args.workload == "region":
        run_region(args, world, rank, P, torch, dist)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

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
              "dataflow": P.ISING_ENGINE_DATAFLOW,
              "persistent_grid": P.ISING_ENGINE_PERSISTENT_GRID,
              "itemflow": P.ISING_ENGINE_ITEMFLOW, "halo": P.ISING_ENGINE_HALO,
              "hub": P.ISING_ENGINE_HUB}[args.engine]

    h = P.ising_create(g.n, g.src, g.dst, g.w, stream=stream)
    P.ising_set_engine(h, engine)
    P.ising_set_halo_sweeps(h, args.halo_sweeps)
    if args.engine in ("auto", "halo"):
        # setup, like ising_create: let the host planner finish so that every
        # timed step runs the engine AUTO settles on (None: no halo plan)
        P.ising_halo_info(h)
    mode = P.ISING_MODE_RACY if args.mode == "racy" else P.ISING_MODE_DET
    colours = P.ising_num_colours(h)
    m = P.ising_num_edges(h)
    nnz = 2 * m
    w_bytes = 1 if np.abs(g.w).max(initial=0) <= 127 else 4
    # the library packs (column, int8 weight) into one int32 when it can
    lib_entry_bytes = 4 if (w_bytes == 1 and g.n < (1 << 24) - 1) else 8
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
    engine_name = {P.ISING_ENGINE_PHASE: "phase", P.ISING_ENGINE_PERSISTENT_GRID: "persistent",
                   P.ISING_ENGINE_DATAFLOW: "dataflow", P.ISING_ENGINE_ITEMFLOW: "itemflow",
                   P.ISING_ENGINE_HALO: "halo", P.ISING_ENGINE_HUB: "hub",
                   P.ISING_ENGINE_USED_BLOCK: "block"}.get(P.ising_engine_used(h), "unknown")
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, world, dist, "cuda")
    if world > 1:
        dist.barrier()
    value = job_throughput(g.n * T * args.steps, world, total_ms / 1e3)

    # roofline of the sweep kernels: algorithmic bytes per sweep / time per sweep
    B = algorithmic_bytes_per_sweep(g.n, nnz, 4 + w_bytes)
    B_lib = algorithmic_bytes_per_sweep(g.n, nnz, lib_entry_bytes)
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
        e2e_t, create_t = [], []
        e2e_engine = None
        for k in range(args.e2e_steps + 1):
            t0 = time.perf_counter()
            with P.ising_create(g.n, src_p, dst_p, w_p, stream=stream) as h2:
                t1 = time.perf_counter()
                P.ising_set_engine(h2, engine)
                P.ising_set_halo_sweeps(h2, args.halo_sweeps)
                P.ising_init_random(h2, seed + k)
                P.ising_anneal(h2, p0=p0, t_total=T, seed=seed + k, stream=stream, mode=mode)
                P.ising_cut(h2)
                P.ising_get_spins(h2, spins_out)
                e2e_engine = P.ising_engine_used(h2)
            dt = time.perf_counter() - t0
            if k > 0:
                e2e_t.append(dt)
                create_t.append(t1 - t0)
        e2e_total = sum(e2e_t)
        e2e_total = max_over_ranks(e2e_total, world, dist, "cuda")
        e2e = {"value": g.n * T * len(e2e_t) * world / e2e_total, "unit": "spin-updates/s",
               "h2d_bytes_per_step": int(3 * 4 * g.m), "d2h_bytes_per_step": int(g.n + 8),
               "ms_per_step": 1e3 * e2e_total / len(e2e_t),
               # a new handle every step: the host graph build (ising_create) is
               # inside the timed region, and a one-shot handle never waits for
               # the halo plan
               "create_ms_per_step": 1e3 * sum(create_t) / len(create_t),
               "engine_used": {P.ISING_ENGINE_PHASE: "phase", P.ISING_ENGINE_PERSISTENT_GRID: "persistent",
                               P.ISING_ENGINE_DATAFLOW: "dataflow", P.ISING_ENGINE_ITEMFLOW: "itemflow",
                               P.ISING_ENGINE_HALO: "halo", P.ISING_ENGINE_HUB: "hub",
                               P.ISING_ENGINE_USED_BLOCK: "block"}.get(e2e_engine, "unknown")}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    halo = P.ising_halo_info(h) if engine_name == "halo" else None
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
            "engine": args.engine, "engine_used": engine_name, "halo": halo,
            "weights": "int8" if w_bytes == 1 else "int32",
            "csr_entry_bytes": lib_entry_bytes,
            "replicas_per_gpu": 1, "parallelism": f"replicas{world}",
            "l2": "512 MiB buffer zeroed between timed steps (outside the events)",
        },
        "sweeps_per_s": T * args.steps * world / (total_ms / 1e3),
        "algorithmic_gbs": achieved,
        "final_cut_mean": float(np.mean(cuts)),
        "roofline": roofline_entry(args, engine_name, T, B, B_lib, achieved, peak, peak_kind,
                                   sweep_s, clocks.summary()),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks.summary(),
    }
    if secondary and world == 1:
        line["secondary"] = run_secondary()
    print(json.dumps(line), flush=True)
    P.ising_destroy(h)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
