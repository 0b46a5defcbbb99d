"""Seeded synthetic graph generators.

This module is shared by the tests, the benchmark, the CPU oracle's callers and
the CUDA path's callers. It only *draws* inputs (edge lists and weights); it
holds none of the annealing arithmetic. Every generator is a pure function of
its arguments and a numpy ``default_rng`` seed.

The shapes stand in for the paper's workloads (Table III): G-set-like
Erdos-Renyi graphs, 2-D toroidal grids (the "torus" rows) and large irregular
random graphs (the custom C1-C7 rows). G-set itself is not reproduced.
"""

from .graphs import (  # noqa: F401
    Graph,
    batched_er_graphs,
    batched_workload,
    BATCHED,
    WARMSTART,
    WARMSTART_BATCHED,
    graph_from_spec,
    warmstart_specs,
    warmstart_workload,
    complete_graph,
    cycle_graph,
    er_graph,
    grid_graph,
    random_small_graph,
    torus_graph,
    draw_weights,
    zipf_config_graph,
    workload,
    WORKLOADS,
)
from .gnn_init import GNN_NUM_PARAMS, gnn_init_params  # noqa: F401
