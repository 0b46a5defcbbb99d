"""ising_energy_csr_static, the entry point that allocates nothing.

Some callers cannot call cudaMalloc: their device memory belongs to a pool they
do not control, they run under a fixed memory budget, or they sit in a loop
where cudaMalloc's host blocking and device synchronisation are not acceptable.
For them the library computes energy and cut of spins on a CSR graph the
caller owns, with its scratch in a fixed device array instead of an
allocation. This test calls it through the C ABI twice in a row and checks
both results against the CPU oracle's energy and cut of the same edge list and
spins (exact integers, so equality). The existing handle-based ising_energy /
ising_cut must agree with both.

This file is named to be collected last.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def caller_csr(g):
    """The caller's own symmetric CSR in its own vertex order: every listed
    edge in both rows (repeats and zero weights are harmless: they add)."""
    rows = np.concatenate([g.src, g.dst]).astype(np.int64)
    cols = np.concatenate([g.dst, g.src]).astype(np.int32)
    ws = np.concatenate([g.w, g.w]).astype(np.int32)
    order = np.argsort(rows, kind="stable")
    counts = np.bincount(rows, minlength=g.n)
    row_ptr = np.zeros(g.n + 1, np.int32)
    row_ptr[1:] = np.cumsum(counts)
    return row_ptr, cols[order], ws[order]


@pytest.mark.parametrize("make", [
    lambda: synth.random_small_graph(3001, 0.004, 21, weights="int8", duplicates=80),
    lambda: synth.torus_graph(300, 4, weights="pm1"),
    # 300,001 rows: 293 chunks of 1024 rows (more than the finishing kernel's
    # 256 threads, so some threads sum several partials) and a ragged last chunk
    lambda: synth.random_small_graph(300001, 6.0 / 300000, 22, weights="int8", duplicates=500),
], ids=["er3001", "torus300", "er300001"])
def test_static_energy_matches_oracle_on_two_calls(make):
    import torch
    from paper_1807_10750_gb300 import _build
    _build.build()
    import paper_1807_10750_gb300 as P

    g = make()
    rp, col, w = caller_csr(g)
    dev = torch.device("cuda")
    rp_d = torch.from_numpy(rp).to(dev)
    col_d = torch.from_numpy(col).to(dev)
    w_d = torch.from_numpy(w).to(dev)
    out = torch.zeros(2, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        for call in range(2):
            s = (rng.integers(0, 2, g.n) * 2 - 1).astype(np.int8)
            H, _, cut = oracle.energy_cut(g.n, g.src, g.dst, g.w, s)
            out.fill_(-12345)
            P.ising_energy_csr_static(g.n, rp_d, col_d, w_d, torch.from_numpy(s).to(dev), out,
                                      stream=stream)
            torch.cuda.synchronize()
            assert tuple(int(x) for x in out.cpu()) == (H, cut), f"call {call}"
            P.ising_set_spins(h, s)
            assert (P.ising_energy(h), P.ising_cut(h)) == (H, cut), f"call {call}"
