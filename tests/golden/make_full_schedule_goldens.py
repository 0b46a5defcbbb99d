"""Write the full-schedule expected results of the large workloads.

Runs the CPU oracle (only ``oracle/`` and the seeded generators of ``synth/``)
over the whole schedule of each large workload and stores, per result, a
SHA-256 of the final spin vector (int8, caller order) with the exact cut and
energy. The GPU tests compare the CUDA path's final spins with these digests;
a mismatch is then localised element by element against a fresh oracle run.

    python tests/golden/make_full_schedule_goldens.py [torus1024] [zipf1m] [batched]

Initial spins are the oracle's Philox stream-1 draw with the workload's seed,
and the anneal uses the same seed (seed 1 for every workload, as in the
workload definitions). The 2^20-vertex power-law workload takes about five
minutes on one core; the batched workload's 8192 anneals run on every core.
"""

from __future__ import annotations

import hashlib
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def spins_digest(s: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(s, dtype=np.int8).tobytes()).hexdigest()


def single(name: str) -> None:
    g, sch = synth.workload(name)
    seed, p0, T = sch["seed"], sch["p0"], sch["sweeps"]
    t0 = time.time()
    s0 = oracle.init_spins(g.n, seed)
    s = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=seed, p0=p0, T=T)
    H, W, cut = oracle.energy_cut(g.n, g.src, g.dst, g.w, s)
    path = os.path.join(HERE, f"full_schedule_{name}.txt")
    with open(path, "w") as f:
        f.write(f"# {name}: oracle.anneal over the whole schedule (written by "
                f"make_full_schedule_goldens.py)\n")
        f.write(f"# n={g.n} edges={g.m} init_seed={seed} seed={seed} p0={p0} T={T}\n")
        f.write("# sha256(final int8 spins, caller order) cut energy\n")
        f.write(f"{spins_digest(s)} {cut} {H}\n")
    print(f"{name}: cut {cut} in {time.time() - t0:.0f} s -> {path}", flush=True)


_GRAPHS = None  # the batched workload's graphs, generated once per worker process


def _batch_instance(args):
    global _GRAPHS
    gi, seed, p0, T, R = args
    if _GRAPHS is None:
        _GRAPHS = synth.batched_workload()[0]
    g = _GRAPHS[gi]
    h = hashlib.sha256()
    cut_sum = 0
    for r in range(R):
        s0 = oracle.init_spins(g.n, seed, instance=gi, replica=r)
        s = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=seed, p0=p0, T=T, instance=gi, replica=r)
        h.update(np.ascontiguousarray(s, dtype=np.int8).tobytes())
        cut_sum += oracle.energy_cut(g.n, g.src, g.dst, g.w, s)[2]
    return gi, g.n, h.hexdigest()[:32], cut_sum


def batched() -> None:
    gs, sch = synth.batched_workload()
    seed, p0, T, R = sch["seed"], sch["p0"], sch["sweeps"], sch["replicas"]
    t0 = time.time()
    jobs = [(gi, seed, p0, T, R) for gi in range(len(gs))]
    # largest instances first so the pool ends together
    jobs.sort(key=lambda j: -gs[j[0]].n)
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        rows = sorted(pool.imap_unordered(_batch_instance, jobs, chunksize=1))
    path = os.path.join(HERE, "full_schedule_batched.txt")
    with open(path, "w") as f:
        f.write("# batched: per instance, oracle.anneal of every replica over the whole schedule "
                "(written by make_full_schedule_goldens.py)\n")
        f.write(f"# instances={len(gs)} replicas={R} init_seed={seed} seed={seed} p0={p0} T={T}\n")
        f.write("# instance n sha256(replica 0..R-1 final spins, concatenated)[:32] sum_of_cuts\n")
        for gi, n, dig, cs in rows:
            f.write(f"{gi} {n} {dig} {cs}\n")
    print(f"batched: {len(rows)} instances in {time.time() - t0:.0f} s -> {path}", flush=True)


def main(argv):
    names = argv or ["torus1024", "zipf1m", "batched"]
    for name in names:
        if name == "batched":
            batched()
        else:
            single(name)


if __name__ == "__main__":
    main(sys.argv[1:])
