"""FP64 oracle of the warm-start graph network (a project addition; the paper
has no learned part).

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's baseline legs are the
only callers; the product package never imports this module and this module
imports nothing from it.

The network (readings G1-G6, restated in the library header):

* G1 normalisation. Edges are merged as the annealer merges them (R7: repeated
  pairs summed, zero sums dropped). d_i = sum_j |w_ij|, c_i = (d_i + 1)^-1/2,
  and the propagation matrix is A_hat = C W C (W the merged signed weights).
* G2 input features of vertex i, given spins s (+-1) of the annealer:
  x_i = [s_i, f_i c_i^2, s_i f_i c_i^2, log(1 + deg_i) / 8, (sum_j w_ij) c_i^2,
  1, 0, 0] with f_i = sum_j w_ij s_j (the local field of Eq. 2) and deg_i the
  number of merged neighbours.
* G3 three message-passing layers, hidden width 64: for l = 0, 1, 2,
  a^l = A_hat h^l, u^l = [h^l, a^l] W_l + b_l, h^(l+1) = relu(u^l), with
  h^0 = x; the logit is z = h^3 w_o + b_o.
* G4 loss against annealer spins y (+-1): L = mean_i softplus(-y_i z_i).
* G5 warm start: s_i = +1 if z_i > 0, -1 if z_i < 0, unchanged if z_i = 0.
* G6 flip bias: q_i = min(255, round(512 * sigmoid(-|z_i|))), the per-vertex
  factor q_i / 128 on the flip threshold of R11.

Storage rounding (optional). The network's stated arithmetic is bf16
operands with fp32 accumulation, so a device computes it with every stored
activation rounded to bf16. `forward` and `backward` take `storage="bf16"`
to apply exactly those roundings, each at the point where the data leaves a
computation as a bf16 operand, and nothing else (all sums stay in float64):

* forward: x = R(x); a^l = R(A_hat h^l); h^(l+1) = R(relu(u^l)); the head
  z = h^3 w_o + b_o is unrounded;
* backward: with dU^l = dh^(l+1) * [u^l > 0], the products that feed the
  tensor cores use R(dU^l): dW_l = X_l^T R(dU^l) and dX_l = R(dU^l) W_l^T;
  db_l sums the unrounded dU^l; the part of dX_l that multiplies a^l is
  rounded before it is propagated back through A_hat: dh^l = dX_l[:, :H] +
  A_hat R(dX_l[:, H:]).

R rounds a value to float32 (nearest) and then to bf16 (nearest, ties to
even), the value a float32 computation stores. The default (`storage=None`)
is the plain float64 network, the definition the rounded form approximates.

Parameters travel as one flat float array in this order (row-major):
W_0 [16, 64], b_0 [64], W_1 [128, 64], b_1 [64], W_2 [128, 64], b_2 [64],
w_o [64], b_o [1] -- 17,665 values. Row k of W_l multiplies feature k of the
concatenation [h^l, a^l]; column j feeds hidden unit j.
"""

from __future__ import annotations

import numpy as np

F_IN = 8
HIDDEN = 64
LAYERS = 3
SHAPES = [("W0", (2 * F_IN, HIDDEN)), ("b0", (HIDDEN,)),
          ("W1", (2 * HIDDEN, HIDDEN)), ("b1", (HIDDEN,)),
          ("W2", (2 * HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("wo", (HIDDEN,)), ("bo", (1,))]
NUM_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat) -> dict:
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.shape == (NUM_PARAMS,)
    out, k = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = flat[k:k + size].reshape(shape)
        k += size
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


class Graph:
    """Merged undirected graph (R7) as a symmetric list of directed entries."""

    def __init__(self, n, src, dst, w):
        src = np.asarray(src, np.int64)
        dst = np.asarray(dst, np.int64)
        w = np.asarray(w, np.int64)
        if np.any(src == dst) or np.any((src < 0) | (src >= n) | (dst < 0) | (dst >= n)):
            raise ValueError("invalid graph")
        lo, hi = np.minimum(src, dst), np.maximum(src, dst)
        key = lo * n + hi
        uk, inv = np.unique(key, return_inverse=True)
        wsum = np.zeros(uk.size, np.int64)
        np.add.at(wsum, inv, w)
        keep = wsum != 0
        uk, wsum = uk[keep], wsum[keep]
        u, v = uk // n, uk % n
        self.n = int(n)
        self.row = np.concatenate([u, v])      # directed entries (row, col, weight)
        self.col = np.concatenate([v, u])
        self.w = np.concatenate([wsum, wsum]).astype(np.float64)
        self.deg = np.bincount(self.row, minlength=n).astype(np.float64)
        self.d = np.bincount(self.row, weights=np.abs(self.w), minlength=n)
        self.wsum = np.bincount(self.row, weights=self.w, minlength=n)
        self.c = 1.0 / np.sqrt(self.d + 1.0)

    def propagate(self, h):
        """A_hat h (G1), summed entry by entry."""
        h = np.asarray(h, np.float64)
        out = np.zeros_like(h)
        coef = self.c[self.row] * self.w * self.c[self.col]
        np.add.at(out, self.row, coef[:, None] * h[self.col])
        return out


def features(G: Graph, s) -> np.ndarray:
    """G2."""
    s = np.asarray(s, np.float64)
    f = np.bincount(G.row, weights=G.w * s[G.col], minlength=G.n)
    c2 = G.c ** 2
    x = np.zeros((G.n, F_IN))
    x[:, 0] = s
    x[:, 1] = f * c2
    x[:, 2] = s * f * c2
    x[:, 3] = np.log1p(G.deg) / 8.0
    x[:, 4] = G.wsum * c2
    x[:, 5] = 1.0
    return x


def to_bf16(v) -> np.ndarray:
    """R: float64 -> float32 (nearest) -> bf16 (nearest, ties to even), as
    float64. Finite inputs only."""
    f = np.asarray(v, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _rounder(storage):
    if storage is None:
        return lambda v: np.asarray(v, np.float64)
    if storage == "bf16":
        return to_bf16
    raise ValueError(f"unknown storage {storage!r}")


def forward(G: Graph, x, params, storage=None) -> tuple[np.ndarray, dict]:
    """G3: logits z and the intermediates the backward pass needs."""
    R = _rounder(storage)
    p = unpack(params) if not isinstance(params, dict) else params
    h = R(x)
    cache = {"X": [], "U": []}
    for l in range(LAYERS):
        a = R(G.propagate(h))
        X = np.concatenate([h, a], axis=1)
        U = X @ p[f"W{l}"] + p[f"b{l}"]
        cache["X"].append(X)
        cache["U"].append(U)
        h = R(np.maximum(U, 0.0))
    cache["h3"] = h
    z = h @ p["wo"] + p["bo"][0]
    return z, cache


def loss(z, y) -> float:
    """G4: mean softplus(-y z)."""
    m = -np.asarray(y, np.float64) * np.asarray(z, np.float64)
    return float(np.mean(np.logaddexp(0.0, m)))


def backward(G: Graph, params, cache, z, y, storage=None) -> np.ndarray:
    """Gradient of G4 with respect to the flat parameters (chain rule through
    G3, written out layer by layer); `cache` comes from `forward` with the
    same `storage`."""
    R = _rounder(storage)
    p = unpack(params) if not isinstance(params, dict) else params
    y = np.asarray(y, np.float64)
    n = z.shape[0]
    # d softplus(-y z) / dz = -y * sigmoid(-y z)
    dz = -y / (1.0 + np.exp(y * z)) / n
    g = {"wo": cache["h3"].T @ dz, "bo": np.array([dz.sum()])}
    dh = dz[:, None] * p["wo"][None, :]
    for l in reversed(range(LAYERS)):
        dU = dh * (cache["U"][l] > 0.0)
        dUr = R(dU)
        g[f"W{l}"] = cache["X"][l].T @ dUr
        g[f"b{l}"] = dU.sum(axis=0)
        if l > 0:
            dX = dUr @ p[f"W{l}"].T
            half = dX.shape[1] // 2
            # a^l = A_hat h^l and A_hat is symmetric
            dh = dX[:, :half] + G.propagate(R(dX[:, half:]))
    return pack(g)


def warm_start(z, s) -> np.ndarray:
    """G5."""
    z = np.asarray(z)
    out = np.array(s, dtype=np.int8, copy=True)
    out[z > 0] = 1
    out[z < 0] = -1
    return out


def flip_bias(z) -> np.ndarray:
    """G6 (computed in the precision of z)."""
    z = np.asarray(z)
    sig = 1.0 / (1.0 + np.exp(np.abs(z)))
    return np.minimum(255, np.rint(512.0 * sig)).astype(np.uint8)
