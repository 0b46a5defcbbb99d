"""Failure detection without a GPU fault: a fault injected from the host
makes a bounded device-side wait run out (a barrier arrival that never comes,
a bulk copy whose barrier expects bytes that never arrive); the kernel
records the timeout and returns, the host reports ISING_ETIMEOUT, and the
CUDA context stays usable for a new handle."""

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


def _context_still_works(P):
    g = synth.random_small_graph(300, 0.05, 4, weights="int8")
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_init_random(h, 1)
        s0 = P.ising_get_spins(h)
        P.ising_anneal(h, p0=0.1, t_total=20, seed=2)
        got = P.ising_get_spins(h)
    assert np.array_equal(got, oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=2, p0=0.1, T=20))


@pytest.mark.parametrize("engine,kind,n", [
    ("grid", "skip_arrival", 20000),
    ("grid", "skip_arrival", 500),
    ("block", "short_copy", 500),
])
def test_injected_fault_reports_timeout(P, engine, kind, n):
    g = synth.random_small_graph(n, 8.0 / n, 6, weights="int8")
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_engine(h, P.ISING_ENGINE_PERSISTENT_GRID if engine == "grid"
                           else P.ISING_ENGINE_PERSISTENT)
        P.ising_debug_fault(h, P.ISING_FAULT_SKIP_ARRIVAL if kind == "skip_arrival"
                            else P.ISING_FAULT_SHORT_COPY, 50_000_000)   # 50 ms
        P.ising_init_random(h, 1)
        P.ising_anneal(h, p0=0.1, t_total=30, seed=3)
        with pytest.raises(P.IsingError) as e:
            P.ising_cut(h)
        assert e.value.code == P.ISING_ETIMEOUT
        # the status is latched in the handle
        with pytest.raises(P.IsingError) as e:
            P.ising_anneal(h, p0=0.1, t_total=30, seed=3)
        assert e.value.code == P.ISING_ETIMEOUT
    _context_still_works(P)


def test_halo_engine_missing_publication_reports_timeout(P):
    # block 0 of the halo engine never publishes its epochs: its neighbour
    # parts' waits run out, every block returns
    g = synth.torus_graph(128, 2, weights="pm1")
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_engine(h, P.ISING_ENGINE_HALO)
        P.ising_debug_fault(h, P.ISING_FAULT_SKIP_ARRIVAL, 50_000_000)   # 50 ms
        P.ising_init_random(h, 1)
        P.ising_anneal(h, p0=0.1, t_total=30, seed=3)
        assert P.ising_engine_used(h) == P.ISING_ENGINE_HALO
        with pytest.raises(P.IsingError) as e:
            P.ising_cut(h)
        assert e.value.code == P.ISING_ETIMEOUT
    _context_still_works(P)


def test_debug_fault_arguments(P):
    g = synth.random_small_graph(50, 0.1, 1)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        for kind, budget in ((7, 0), (P.ISING_FAULT_NONE, 61 * 10 ** 9)):
            with pytest.raises(P.IsingError) as e:
                P.ising_debug_fault(h, kind, budget)
            assert e.value.code == P.ISING_EINVAL
        # no fault: a short budget changes nothing for a healthy anneal
        P.ising_debug_fault(h, P.ISING_FAULT_NONE, 50_000_000)
        P.ising_init_random(h, 1)
        s0 = P.ising_get_spins(h)
        P.ising_anneal(h, p0=0.1, t_total=20, seed=2)
        got = P.ising_get_spins(h)
    assert np.array_equal(got, oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=2, p0=0.1, T=20))
