"""The hub engine (ISING_ENGINE_HUB) against the CPU oracle, bit for bit.

The engine runs every hub class (vertices with at least ISING_HUB_DEGREE
neighbours, coloured and swept first) in one block with the hubs' fields in
shared memory, and the other classes on the rest of the GPU. These cases
cover what that split can get wrong: a hub class wider than the block (it is
decided in steps of 512), hubs without hub neighbours, int32 weights, a graph
whose every vertex is a hub (no other class), several calls that resume the
schedule, the flip bias, and a failure injected at a grid barrier.
"""

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


def run_hub(P, g, s0, *, seed, p0, T, t_begin=0, sweeps=None, flags=0, bias=None, calls=1):
    """Anneal with the hub engine, split into `calls` consecutive calls."""
    if sweeps is None:
        sweeps = T - t_begin
    with P.ising_create(g.n, g.src, g.dst, g.w, flags=flags) as h:
        P.ising_set_engine(h, P.ISING_ENGINE_HUB)
        P.ising_set_spins(h, s0)
        if bias is not None:
            P.ising_set_flip_bias(h, bias)
        cuts = np.linspace(t_begin, t_begin + sweeps, calls + 1).astype(int)
        for a, b in zip(cuts[:-1], cuts[1:]):
            if b > a:
                P.ising_anneal(h, p0=p0, t_total=T, t_begin=int(a), sweeps=int(b - a), seed=seed)
                assert P.ising_engine_used(h) == P.ISING_ENGINE_HUB
        return P.ising_get_spins(h), P.ising_energy(h), P.ising_cut(h)


def check_hub(P, g, *, seed, p0, T, t_begin=0, sweeps=None, flags=0, bias=None, calls=1, s0=None):
    if s0 is None:
        s0 = oracle.init_spins(g.n, seed + 77)
    want = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=seed, p0=p0, T=T, t_begin=t_begin,
                         sweeps=sweeps, bias=bias)
    got, H, cut = run_hub(P, g, s0, seed=seed, p0=p0, T=T, t_begin=t_begin, sweeps=sweeps,
                          flags=flags, bias=bias, calls=calls)
    mism = np.nonzero(got != want)[0]
    assert mism.size == 0, f"{mism.size} spins differ, first at {mism[:8]}"
    assert (H, cut) == oracle.energy_cut(g.n, g.src, g.dst, g.w, want)[::2]
    return got


def hub_count(g):
    C, col = oracle.colouring(g.n, g.src, g.dst, g.w)
    deg = np.zeros(g.n, np.int64)
    pairs = set()
    for u, v in zip(g.src.tolist(), g.dst.tolist()):
        pairs.add((min(u, v), max(u, v)))
    for u, v in pairs:
        deg[u] += 1
        deg[v] += 1
    return int((deg >= 256).sum())


def independent_hubs(hubs, leaves, degree, seed, weights="int8"):
    """`hubs` mutually non-adjacent hubs, each joined to `degree` random
    leaves: every hub lands in hub class 0, wider than one decision step."""
    rng = np.random.default_rng(seed)
    src = np.repeat(np.arange(hubs, dtype=np.int64), degree)
    dst = hubs + np.concatenate([rng.choice(leaves, degree, replace=False) for _ in range(hubs)])
    noise = synth.er_graph(leaves, 3.0 / leaves, seed + 1, weights=weights)
    src = np.concatenate([src, noise.src + hubs])
    dst = np.concatenate([dst, noise.dst + hubs])
    w = synth.draw_weights(weights, src.size, rng)
    return synth.Graph(hubs + leaves, src.astype(np.int32), dst.astype(np.int32), w)


def test_power_law_graph_uses_hub_engine_and_matches(P):
    g = synth.zipf_config_graph(30000, 2.0, 3, 3000, 11)
    assert hub_count(g) >= 20
    check_hub(P, g, seed=5, p0=0.15, T=80)


def test_hub_class_wider_than_a_decision_step(P):
    g = independent_hubs(1100, 40000, 300, 3)
    C, col = oracle.colouring(g.n, g.src, g.dst, g.w)
    assert int((col[:1100] == 0).sum()) == 1100
    check_hub(P, g, seed=9, p0=0.2, T=25)


def test_hubs_with_int32_weights_and_forced_split_layout(P):
    g = synth.zipf_config_graph(20000, 2.0, 3, 2500, 12)
    g32 = synth.Graph(g.n, g.src, g.dst, (g.w * 91).astype(np.int32))
    check_hub(P, g32, seed=4, p0=0.1, T=30)
    check_hub(P, g, seed=4, p0=0.1, T=30, flags=P.ISING_CREATE_WEIGHTS_I32)


def test_every_vertex_a_hub(P):
    # K_300: 300 hub classes of one vertex, no other class
    g = synth.complete_graph(300, 2, weights="int8")
    check_hub(P, g, seed=6, p0=0.3, T=40)


def test_hub_engine_resumes_across_calls(P):
    g = synth.zipf_config_graph(25000, 2.0, 3, 3000, 13)
    check_hub(P, g, seed=8, p0=0.1, T=90, calls=5)
    check_hub(P, g, seed=8, p0=0.1, T=90, t_begin=70, calls=3)


def test_hub_engine_with_flip_bias(P):
    g = synth.zipf_config_graph(20000, 2.0, 3, 3000, 14)
    q = np.random.default_rng(2).integers(0, 256, g.n).astype(np.uint8)
    check_hub(P, g, seed=2, p0=0.3, T=40, bias=q)


def test_hub_engine_every_spin_flipping(P):
    # p0 = 1: almost every hub changes in the first sweeps, so every class
    # pushes along most of its hubs' rows (the small classes' shared pushes,
    # the 128-entry push tasks and their list, the deferred queue at its
    # fullest)
    g = synth.zipf_config_graph(40000, 2.0, 3, 4000, 19)
    check_hub(P, g, seed=11, p0=1.0, T=12)


def test_hub_engine_long_run(P):
    # many chain steps with changes early and none late
    g = synth.zipf_config_graph(50000, 2.1, 4, 5000, 15)
    check_hub(P, g, seed=1, p0=0.1, T=300)


def test_hub_engine_missing_arrival_reports_timeout(P):
    g = synth.zipf_config_graph(20000, 2.0, 3, 3000, 16)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_engine(h, P.ISING_ENGINE_HUB)
        P.ising_debug_fault(h, P.ISING_FAULT_SKIP_ARRIVAL, 50_000_000)   # 50 ms per wait
        P.ising_init_random(h, 1)
        P.ising_anneal(h, p0=0.1, t_total=30, seed=3)
        with pytest.raises(P.IsingError) as e:
            P.ising_cut(h)
        assert e.value.code == P.ISING_ETIMEOUT
    # the context stays usable
    g2 = synth.zipf_config_graph(20000, 2.0, 3, 3000, 17)
    check_hub(P, g2, seed=3, p0=0.1, T=10)


def test_hub_engine_without_a_shared_memory_map(P):
    # 2^21 vertices: the spin map (256 KiB) does not fit in a block's shared
    # memory, so the workers read the global map
    g = synth.zipf_config_graph(1 << 21, 2.5, 3, 3000, 18)  # ~2000 hubs
    check_hub(P, g, seed=3, p0=0.1, T=2000, sweeps=4)
