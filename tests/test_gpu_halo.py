"""The halo engine (ISING_ENGINE_HALO) against the oracle: deterministic
anneals bit for bit, on graphs it takes -- lattices with 2, 3 or 4 colour
classes, a 3-D torus, a diluted torus, disconnected tori -- for several sweeps
per exchange, epochs cut short at the end of a call, resumed calls, replicas
and a flip bias; and the fallback when no plan exists."""

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


def torus3d(L, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(L),) * 3, indexing="ij")
    v = ((z * L + y) * L + x).ravel()
    nbrs = [((z * L + y) * L + (x + 1) % L), ((z * L + (y + 1) % L) * L + x), ((((z + 1) % L) * L + y) * L + x)]
    src = np.concatenate([v] * 3)
    dst = np.concatenate([a.ravel() for a in nbrs])
    w = synth.draw_weights("int8", src.size, rng)
    return synth.Graph(L ** 3, src.astype(np.int32), dst.astype(np.int32), w)


def diluted_torus(L, keep, seed):
    g = synth.torus_graph(L, seed, weights="int8")
    m = np.random.default_rng(seed).random(g.src.size) < keep
    return synth.Graph(g.n, g.src[m], g.dst[m], g.w[m])


def two_tori():
    a = synth.torus_graph(90, 5, weights="int8")
    b = synth.torus_graph(70, 6, weights="pm1", Ly=51)
    return synth.Graph(a.n + b.n, np.concatenate([a.src, b.src + a.n]).astype(np.int32),
                       np.concatenate([a.dst, b.dst + a.n]).astype(np.int32),
                       np.concatenate([a.w, b.w]).astype(np.int32))


# every graph has at least 64 vertices per SM, at most 4 colours and short rows
HALO_GRAPHS = {
    "torus128_pm1": lambda: synth.torus_graph(128, 1, weights="pm1"),
    "torus_odd_int8": lambda: synth.torus_graph(127, 2, weights="int8", Ly=101),
    "torus3d_24": lambda: torus3d(24, 3),
    "diluted_torus": lambda: diluted_torus(160, 0.7, 4),
    "two_tori": two_tori,
}


def run_halo(P, g, s0, *, S, seed, p0, T, splits=(None,), replica=0, bias=None):
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_engine(h, P.ISING_ENGINE_HALO)
        P.ising_set_halo_sweeps(h, S)
        P.ising_set_spins(h, s0)
        if bias is not None:
            P.ising_set_flip_bias(h, bias)
        t = 0
        for k in splits:
            P.ising_anneal(h, p0=p0, t_total=T, t_begin=t, sweeps=k, seed=seed, replica=replica)
            t = T if k is None else t + k
        info = P.ising_halo_info(h)
        return P.ising_get_spins(h), P.ising_cut(h), P.ising_engine_used(h), info


@pytest.mark.parametrize("S", [0, 1, 2, 3])
@pytest.mark.parametrize("name", sorted(HALO_GRAPHS))
def test_halo_bit_exact(P, name, S):
    g = HALO_GRAPHS[name]()
    s0 = oracle.init_spins(g.n, 11)
    T = 37   # not a multiple of 2 or 3: the last epoch is cut short
    got, cut, used, info = run_halo(P, g, s0, S=S, seed=6, p0=0.15, T=T)
    want = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=6, p0=0.15, T=T)
    K, _ = P.ising_plan_colouring(g.n, g.src, g.dst, g.w)
    if S * K <= 16:
        assert used == P.ISING_ENGINE_HALO
        assert info["sweeps_per_exchange"] == S if S else info["sweeps_per_exchange"] in (1, 2)
    mism = np.nonzero(got != want)[0]
    assert mism.size == 0, f"{mism.size} spins differ, first at {mism[:8]}"
    assert cut == oracle.energy_cut(g.n, g.src, g.dst, g.w, want)[2]


@pytest.mark.parametrize("name", ["torus128_pm1", "torus_odd_int8"])
def test_halo_resumed_calls_replica_and_bias(P, name):
    g = HALO_GRAPHS[name]()
    s0 = oracle.init_spins(g.n, 2)
    q = np.random.default_rng(3).integers(0, 256, size=g.n).astype(np.uint8)
    T = 50
    got, _, used, _ = run_halo(P, g, s0, S=2, seed=9, p0=0.2, T=T, splits=(17, 0, 1, None),
                               replica=5, bias=q)
    assert used == P.ISING_ENGINE_HALO
    want = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=9, p0=0.2, T=T, replica=5, bias=q)
    assert np.array_equal(got, want)


def test_halo_many_sweeps(P):
    # 400 sweeps: 200 exchanges, parts running ahead of one another
    g = HALO_GRAPHS["diluted_torus"]()
    s0 = oracle.init_spins(g.n, 5)
    got, _, used, _ = run_halo(P, g, s0, S=0, seed=2, p0=0.1, T=400)
    assert used == P.ISING_ENGINE_HALO
    assert np.array_equal(got, oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=2, p0=0.1, T=400))


def test_halo_fallbacks(P):
    # no plan (S * K > 16, too few vertices, too many colours), racy and
    # N-flip anneals: another engine runs, with the same result
    g = HALO_GRAPHS["torus_odd_int8"]()
    K, _ = P.ising_plan_colouring(g.n, g.src, g.dst, g.w)
    s0 = oracle.init_spins(g.n, 3)
    got, _, used, info = run_halo(P, g, s0, S=16 // K + 1, seed=1, p0=0.1, T=20)
    assert used == P.ISING_ENGINE_ITEMFLOW and info is None
    assert np.array_equal(got, oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=1, p0=0.1, T=20))
    for small in (synth.torus_graph(96, 2, weights="pm1"), synth.random_small_graph(20000, 4e-4, 2)):
        with P.ising_create(small.n, small.src, small.dst, small.w) as h:
            assert P.ising_halo_info(h) is None
            P.ising_set_engine(h, P.ISING_ENGINE_HALO)
            P.ising_init_random(h, 1)
            P.ising_anneal(h, p0=0.1, t_total=5, seed=1)
            assert P.ising_engine_used(h) != P.ISING_ENGINE_HALO
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_engine(h, P.ISING_ENGINE_HALO)
        P.ising_init_random(h, 1)
        P.ising_anneal(h, p0=0.1, t_total=5, seed=1, mode=P.ISING_MODE_RACY)
        assert P.ising_engine_used(h) == P.ISING_ENGINE_PERSISTENT_GRID
        P.ising_anneal(h, t_total=5, seed=1, kind=P.ISING_SCHED_NFLIP, n0=20)
        assert P.ising_engine_used(h) == P.ISING_ENGINE_PERSISTENT_GRID
        with pytest.raises(P.IsingError) as e:
            P.ising_set_halo_sweeps(h, 17)
        assert e.value.code == P.ISING_EINVAL


def test_auto_does_not_wait_for_the_plan_and_destroy_cancels_it(P):
    # AUTO's first call never plans and later calls run another engine while
    # the host planner is busy; either way the result is the oracle's, and
    # destroying the handle stops the planner
    import time
    g = synth.torus_graph(512, 3, weights="pm1")
    s0 = oracle.init_spins(g.n, 4)
    want = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=5, p0=0.1, T=6)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_spins(h, s0)
        P.ising_anneal(h, p0=0.1, t_total=6, seed=5, sweeps=2)   # the first call never plans
        assert P.ising_engine_used(h) == P.ISING_ENGINE_ITEMFLOW
        P.ising_anneal(h, p0=0.1, t_total=6, seed=5, t_begin=2)  # starts the planner
        assert P.ising_engine_used(h) in (P.ISING_ENGINE_HALO, P.ISING_ENGINE_ITEMFLOW)
        assert np.array_equal(P.ising_get_spins(h), want)
    t0 = time.perf_counter()
    h = P.ising_create(g.n, g.src, g.dst, g.w)
    P.ising_init_random(h, 1)
    for _ in range(2):
        P.ising_anneal(h, p0=0.1, t_total=4, seed=1)
    P.ising_destroy(h)
    assert time.perf_counter() - t0 < 5.0


def test_halo_info_and_auto_choice(P):
    # 147,456 vertices, about 970 per part: S = 2 repeats about 1.4x the work
    import torch
    g = synth.torus_graph(384, 1, weights="pm1")
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        info = P.ising_halo_info(h)
        assert info["parts"] == torch.cuda.get_device_properties(0).multi_processor_count
        assert info["sweeps_per_exchange"] == 2 and 1.0 <= info["work_ratio"] <= 1.6
        P.ising_init_random(h, 1)
        P.ising_anneal(h, p0=0.1, t_total=10, seed=1)
        assert P.ising_engine_used(h) == P.ISING_ENGINE_HALO
        P.ising_set_halo_sweeps(h, 1)
        assert P.ising_halo_info(h)["sweeps_per_exchange"] == 1
    # 66 vertices per part: too much repeated work for AUTO, item dataflow runs
    g = synth.torus_graph(100, 1, weights="pm1")
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        assert P.ising_halo_info(h)["work_ratio"] > 1.6
        P.ising_init_random(h, 1)
        P.ising_anneal(h, p0=0.1, t_total=10, seed=1)
        assert P.ising_engine_used(h) == P.ISING_ENGINE_ITEMFLOW
