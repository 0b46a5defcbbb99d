"""Batched annealing (many instances x replicas in one persistent kernel):
every instance and replica must match the oracle's single-graph anneal keyed by
that instance and replica, bit for bit."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_1807_10750_gb300 import _build
    _build.build()
    import paper_1807_10750_gb300 as P
    return P


def small_batch():
    gs = []
    for k in range(10):
        n = 30 + 41 * k
        g = synth.random_small_graph(n, 6.0 / n, 100 + k, weights="int8" if k % 2 else "pm1",
                                     duplicates=k)
        gs.append(g)
    gs.append(synth.Graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32)))
    gs.append(synth.torus_graph(8, 3, weights="pm1"))
    # a star whose hub row sums |w| to more than 255 (the instance takes the
    # per-replica loop instead of byte-lane sums), plus a few extra edges
    rng = np.random.default_rng(5)
    leaves = np.arange(1, 61, dtype=np.int32)
    src = np.concatenate([np.zeros(60, np.int32), leaves[:-1]])
    dst = np.concatenate([leaves, leaves[1:]])
    w = (rng.integers(5, 9, size=src.size) * rng.choice([-1, 1], size=src.size)).astype(np.int32)
    gs.append(synth.Graph(61, src, dst, w))
    # power-law instances: rows longer than byte lanes can sum are decided by
    # a whole warp (int8 weights: more than 31 entries; +-1 weights: more
    # than 255), and weights up to |w| = 96 take the per-replica sums
    gs.append(synth.zipf_config_graph(3000, 2.0, 3, 600, 31, weights="int8"))
    gs.append(synth.zipf_config_graph(4000, 2.0, 3, 900, 32, weights="pm1"))
    g = synth.random_small_graph(200, 0.05, 33, weights="int8")
    gs.append(synth.Graph(g.n, g.src, g.dst, (g.w * 12).astype(np.int32)))
    return gs


def oracle_run(g, gi, r, *, init_seed, seed, p0, T, t_begin=0, sweeps=None, s0=None):
    if s0 is None:
        s0 = oracle.init_spins(g.n, init_seed, instance=gi, replica=r)
    return oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=seed, p0=p0, T=T, t_begin=t_begin,
                         sweeps=sweeps, instance=gi, replica=r)


@pytest.mark.parametrize("block", [128, 256, 512])
def test_batch_bit_exact_every_instance_and_replica(P, block):
    gs = small_batch()
    with P.ising_batch_create([(g.n, g.src, g.dst, g.w) for g in gs], replicas=8) as b:
        P.ising_batch_set_block(b, block)
        P.ising_batch_init_random(b, 77)
        for gi, g in enumerate(gs):
            for r in (0, 5):
                assert np.array_equal(P.ising_batch_get_spins(b, gi, r),
                                      oracle.init_spins(g.n, 77, instance=gi, replica=r))
        P.ising_batch_anneal(b, p0=0.15, t_total=60, seed=9)
        cuts = P.ising_batch_cuts(b)
        for gi, g in enumerate(gs):
            for r in range(8):
                want = oracle_run(g, gi, r, init_seed=77, seed=9, p0=0.15, T=60)
                got = P.ising_batch_get_spins(b, gi, r)
                assert np.array_equal(got, want), (gi, r)
                assert cuts[gi, r] == oracle.energy_cut(g.n, g.src, g.dst, g.w, want)[2]


def test_batch_split_anneal_equals_whole_and_set_spins(P):
    gs = small_batch()[:5]
    rng = np.random.default_rng(4)
    warm = [(rng.integers(0, 2, g.n) * 2 - 1).astype(np.int8) for g in gs]
    with P.ising_batch_create([(g.n, g.src, g.dst, g.w) for g in gs], replicas=3) as b:
        P.ising_batch_init_random(b, 5)
        for gi in range(len(gs)):
            P.ising_batch_set_spins(b, gi, 1, warm[gi])
        P.ising_batch_anneal(b, p0=0.2, t_total=40, seed=3, sweeps=13)
        P.ising_batch_anneal(b, p0=0.2, t_total=40, seed=3, t_begin=13)
        for gi, g in enumerate(gs):
            for r in range(3):
                s0 = warm[gi] if r == 1 else None
                want = oracle_run(g, gi, r, init_seed=5, seed=3, p0=0.2, T=40, s0=s0)
                assert np.array_equal(P.ising_batch_get_spins(b, gi, r), want), (gi, r)


@pytest.mark.parametrize("row_split", [1, 2, 4])
@pytest.mark.parametrize("tail", [0, 32])
def test_batch_every_tuning_is_bit_exact(P, row_split, tail):
    # the autotuner's knobs change only the schedule of the work, never the
    # result: threads sharing a row, one-warp tail classes
    gs = small_batch()
    with P.ising_batch_create([(g.n, g.src, g.dst, g.w) for g in gs], replicas=8) as b:
        P.ising_batch_set_tuning(b, 256, row_split, tail)
        P.ising_batch_init_random(b, 41)
        P.ising_batch_anneal(b, p0=0.15, t_total=40, seed=6)
        for gi, g in enumerate(gs):
            for r in (0, 3, 7):
                want = oracle_run(g, gi, r, init_seed=41, seed=6, p0=0.15, T=40)
                assert np.array_equal(P.ising_batch_get_spins(b, gi, r), want), (gi, r)


def test_batch_autotune_keeps_spins(P):
    gs = small_batch()
    with P.ising_batch_create([(g.n, g.src, g.dst, g.w) for g in gs], replicas=8) as b:
        P.ising_batch_init_random(b, 1)
        before = [P.ising_batch_get_spins(b, gi, 7) for gi in range(len(gs))]
        block = P.ising_batch_autotune(b, probe_sweeps=5)
        assert block in (128, 256, 512)
        assert P.ising_batch_info(b)["block"] == block
        tune = P.ising_batch_tuning(b)
        assert tune["block"] == block and tune["row_split"] in (1, 2, 4) and tune["tail"] in (0, 32)
        assert all(ms > 0 for ms in tune["probe_ms"])
        for gi in range(len(gs)):
            assert np.array_equal(P.ising_batch_get_spins(b, gi, 7), before[gi])


def test_batch_config_shape_sample_bit_exact(P):
    # Instances shaped like the large batched workload (n log-uniform in
    # [500, 20000], mean degree 10, +-1 weights, 8 replicas): a sample of
    # (instance, replica) pairs over the first sweeps of a 1000-sweep schedule.
    gs = synth.batched_er_graphs(24, 500, 20000, 10.0, 11, weights="pm1")
    with P.ising_batch_create([(g.n, g.src, g.dst, g.w) for g in gs], replicas=8) as b:
        P.ising_batch_init_random(b, 2)
        P.ising_batch_anneal(b, p0=0.1, t_total=1000, seed=8, sweeps=25)
        for gi, r in [(0, 0), (3, 7), (11, 2), (17, 5), (23, 3)]:
            g = gs[gi]
            want = oracle_run(g, gi, r, init_seed=2, seed=8, p0=0.1, T=1000, sweeps=25)
            assert np.array_equal(P.ising_batch_get_spins(b, gi, r), want), (gi, r)


def test_batch_rejects_bad_input(P):
    g = synth.cycle_graph(6)
    with pytest.raises(P.IsingError) as e:
        P.ising_batch_create([(g.n, g.src, g.dst, g.w)], replicas=9)
    assert e.value.code == P.ISING_EINVAL
    with pytest.raises(P.IsingError) as e:
        P.ising_batch_create([(g.n, g.src, g.dst, (g.w * 200).astype(np.int32))], replicas=2)
    assert e.value.code == P.ISING_ERANGE
    with pytest.raises(P.IsingError) as e:
        P.ising_batch_create([(3, np.array([0]), np.array([0]), np.array([1]))], replicas=2)
    assert e.value.code == P.ISING_EINVAL
