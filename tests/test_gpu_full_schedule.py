"""Bit-exactness over the whole schedule of the large workloads.

The expected results in tests/golden/full_schedule_*.txt were written by
tests/golden/make_full_schedule_goldens.py, which runs only the CPU oracle:
a SHA-256 of the final spins with the exact cut and energy, after
 * the 1024 x 1024 torus, 2000 sweeps;
 * the 2^20-vertex power-law graph, 2000 sweeps;
 * every instance and replica of the batched workload (1024 graphs, 8
   replicas), 1000 sweeps.
Each deterministic engine that can take the graph must reproduce them. When a
digest differs, the test localises the difference against a fresh oracle run
(the whole run where that takes seconds, else the first sweeps) and reports
the first differing vertices.

The racy mode (no order inside a sweep) is judged by cut only: on the torus
its mean cut over 8 seeds must reach 0.98 of the deterministic mean.
"""

import hashlib
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_1807_10750_gb300 import _build
    _build.build()
    import paper_1807_10750_gb300 as P
    return P


def read_single(name):
    with open(os.path.join(GOLDEN, f"full_schedule_{name}.txt")) as f:
        rows = [ln.split() for ln in f if not ln.startswith("#")]
    digest, cut, energy = rows[0]
    return digest, int(cut), int(energy)


def digest(s):
    return hashlib.sha256(np.ascontiguousarray(s, dtype=np.int8).tobytes()).hexdigest()


ENGINE_NAMES = {"auto": "ISING_ENGINE_AUTO", "halo": "ISING_ENGINE_HALO",
                "itemflow": "ISING_ENGINE_ITEMFLOW", "persistent_grid": "ISING_ENGINE_PERSISTENT_GRID",
                "hub": "ISING_ENGINE_HUB"}


def gpu_full(P, g, sch, engine, sweeps=None):
    seed, p0, T = sch["seed"], sch["p0"], sch["sweeps"]
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_engine(h, getattr(P, ENGINE_NAMES[engine]))
        P.ising_init_random(h, seed)
        P.ising_anneal(h, p0=p0, t_total=T, seed=seed, sweeps=sweeps)
        return P.ising_get_spins(h), P.ising_cut(h), P.ising_energy(h), P.ising_engine_used(h)


def localise(P, g, sch, engine, sweeps):
    """First vertices where the engine and a fresh oracle run differ after
    `sweeps` sweeps of the schedule."""
    got = gpu_full(P, g, sch, engine, sweeps=sweeps)[0]
    s0 = oracle.init_spins(g.n, sch["seed"])
    want = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=sch["seed"], p0=sch["p0"],
                         T=sch["sweeps"], sweeps=sweeps)
    bad = np.nonzero(got != want)[0]
    return f"after {sweeps} sweeps {bad.size} spins differ from the oracle, first at {bad[:8].tolist()}"


@pytest.mark.parametrize("engine", ["auto", "halo", "itemflow", "persistent_grid"])
def test_torus1024_full_schedule(P, engine):
    g, sch = synth.workload("torus1024")
    want_digest, want_cut, want_energy = read_single("torus1024")
    s, cut, energy, used = gpu_full(P, g, sch, engine)
    if digest(s) != want_digest:
        pytest.fail(f"{engine} (ran {used}): final spins differ; " +
                    localise(P, g, sch, engine, sch["sweeps"]))
    assert (cut, energy) == (want_cut, want_energy)


@pytest.mark.parametrize("engine", ["auto", "hub", "persistent_grid"])
def test_zipf1m_full_schedule(P, engine):
    g, sch = synth.workload("zipf1m")
    want_digest, want_cut, want_energy = read_single("zipf1m")
    s, cut, energy, used = gpu_full(P, g, sch, engine)
    if engine == "auto":
        assert used == P.ISING_ENGINE_HUB
    if digest(s) != want_digest:
        pytest.fail(f"{engine} (ran {used}): final spins differ; " + localise(P, g, sch, engine, 20))
    assert (cut, energy) == (want_cut, want_energy)


def test_batched_full_schedule_every_instance_and_replica(P):
    gs, sch = synth.batched_workload()
    seed, p0, T, R = sch["seed"], sch["p0"], sch["sweeps"], sch["replicas"]
    with open(os.path.join(GOLDEN, "full_schedule_batched.txt")) as f:
        rows = [ln.split() for ln in f if not ln.startswith("#")]
    assert len(rows) == len(gs)
    with P.ising_batch_create([(g.n, g.src, g.dst, g.w) for g in gs], replicas=R) as b:
        P.ising_batch_autotune(b, probe_sweeps=10)
        P.ising_batch_init_random(b, seed)
        P.ising_batch_anneal(b, p0=p0, t_total=T, seed=seed)
        cuts = P.ising_batch_cuts(b)
        bad = []
        for gi, n, dig, cut_sum in rows:
            gi = int(gi)
            assert gs[gi].n == int(n)
            h = hashlib.sha256()
            for r in range(R):
                h.update(np.ascontiguousarray(P.ising_batch_get_spins(b, gi, r), np.int8).tobytes())
            if h.hexdigest()[:32] != dig or int(cuts[gi].sum()) != int(cut_sum):
                bad.append(gi)
        if bad:
            gi = bad[0]
            g = gs[gi]
            detail = []
            for r in range(R):
                s0 = oracle.init_spins(g.n, seed, instance=gi, replica=r)
                want = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=seed, p0=p0, T=T,
                                     instance=gi, replica=r)
                diff = np.nonzero(P.ising_batch_get_spins(b, gi, r) != want)[0]
                detail.append(f"replica {r}: {diff.size} differ {diff[:4].tolist()}")
            pytest.fail(f"{len(bad)} instances differ, first {gi}: " + "; ".join(detail))


def test_torus1024_racy_cut_against_deterministic_over_8_seeds(P):
    g, sch = synth.workload("torus1024")
    det, racy = [], []
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        for seed in range(1, 9):
            for mode, out in ((P.ISING_MODE_DET, det), (P.ISING_MODE_RACY, racy)):
                P.ising_init_random(h, seed)
                P.ising_anneal(h, p0=sch["p0"], t_total=sch["sweeps"], seed=seed, mode=mode)
                out.append(P.ising_cut(h))
    assert np.mean(racy) >= 0.98 * np.mean(det), (np.mean(racy), np.mean(det))
