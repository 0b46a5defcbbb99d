"""Seeded initial parameters of the warm-start graph network.

Glorot-uniform weight matrices, zero biases, in the flat layout of the
library header: W_0 [16, 64], b_0, W_1 [128, 64], b_1, W_2 [128, 64], b_2,
w_o [64], b_o [1]. Only random draws live here; the network's arithmetic is
elsewhere.
"""

from __future__ import annotations

import numpy as np

GNN_SHAPES = [(16, 64), (64,), (128, 64), (64,), (128, 64), (64,), (64,), (1,)]
GNN_NUM_PARAMS = sum(int(np.prod(s)) for s in GNN_SHAPES)


def gnn_init_params(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for k, shape in enumerate(GNN_SHAPES):
        if len(shape) == 2:
            lim = np.sqrt(6.0 / (shape[0] + shape[1]))
            parts.append(rng.uniform(-lim, lim, size=shape).ravel())
        elif k == 6:                      # the output weights w_o
            lim = np.sqrt(6.0 / (shape[0] + 1))
            parts.append(rng.uniform(-lim, lim, size=shape))
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)
