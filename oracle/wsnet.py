"""Plain FP64 reference of the learned warm-start network (test infrastructure).

TEST INFRASTRUCTURE ONLY -- imported by tests and by the smoke check, never by
the product library.  The paper has no learned component: its warm start
(Section 3.4) reuses a previous solution.  This network is the project's
addition, which proposes initial prices and node angles for the message
passing iteration; the iteration itself is unchanged and runs to the same
tolerance, so its own stopping test still certifies the result.

The network maps node features to node outputs independently at every time
step t, with the same weights at every step.  Rows are ``r = t * N + n``.

* layer 0:      H0 = relu(X W0 + b0)                    (F -> 64)
* layers 1..3:  H' = relu(H Ws + (A H) Wn + b)           (64 -> 64)
* output:       Y  = H3 Wo + bo                          (64 -> 2)

``A`` is the susceptance-weighted neighbour average over the bus graph:
``(A H)[t, n] = sum_{lines l at n} w_{l,n} H[t, other end of l]`` with
``w_{l,n} = b_l / sum_{lines at n} b``; a node without lines gets 0.  The
loss is ``mean_r sum_o c_o (Y[r, o] - Y*[r, o])^2``.

Weights are kept as FP32 masters and used rounded to bfloat16 (the GPU
stores them in bfloat16 and accumulates in FP32); this reference rounds the
same way and then computes in FP64.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64
N_OUT = 2
N_MP = 3  # message-passing layers


def param_shapes(n_features):
    """Parameter order: W0, b0, then (Ws, Wn, b) per message-passing layer, Wo, bo."""
    shapes = [(n_features, HIDDEN), (HIDDEN,)]
    for _ in range(N_MP):
        shapes += [(HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN,)]
    shapes += [(HIDDEN, N_OUT), (N_OUT,)]
    return shapes


def init_params(n_features, seed):
    """He-uniform weights, zero biases (FP32 masters)."""
    rng = np.random.default_rng(seed)
    out = []
    for shp in param_shapes(n_features):
        if len(shp) == 2:
            lim = np.sqrt(6.0 / shp[0])
            out.append(rng.uniform(-lim, lim, size=shp).astype(np.float32))
        else:
            out.append(np.zeros(shp, np.float32))
    return out


def bf16(x):
    """Round FP32 values to bfloat16 (round to nearest even), returned as FP64."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def neighbour_matrix(n_nodes, line_from, line_to, line_b):
    """Dense ``A`` (N x N) of the susceptance-weighted neighbour average."""
    A = np.zeros((n_nodes, n_nodes))
    bsum = np.zeros(n_nodes)
    for f, t, b in zip(line_from, line_to, line_b):
        bsum[f] += b
        bsum[t] += b
    for f, t, b in zip(line_from, line_to, line_b):
        A[f, t] += b / bsum[f]
        A[t, f] += b / bsum[t]
    return A


class WarmStartNet:
    """Forward and backward passes of the network in FP64."""

    def __init__(self, n_nodes, line_from, line_to, line_b, T):
        self.N, self.T = int(n_nodes), int(T)
        self.A = neighbour_matrix(n_nodes, line_from, line_to, line_b)

    def _agg(self, H):
        # rows t * N + n: apply A per time step
        Hr = H.reshape(self.T, self.N, -1)
        return np.einsum("nm,tmc->tnc", self.A, Hr).reshape(H.shape)

    def _agg_t(self, G):
        Gr = G.reshape(self.T, self.N, -1)
        return np.einsum("mn,tmc->tnc", self.A, Gr).reshape(G.shape)

    @staticmethod
    def _weights(params, round_bf16):
        return [bf16(p) if (p.ndim == 2 and round_bf16) else np.asarray(p, np.float64) for p in params]

    def forward(self, params, X, keep=False, round_bf16=True):
        w = self._weights(params, round_bf16)
        X = np.asarray(X, np.float64)
        Z0 = X @ w[0] + w[1]
        H = np.maximum(Z0, 0.0)
        cache = [(X, Z0)]
        for l in range(N_MP):
            Ws, Wn, b = w[2 + 3 * l], w[3 + 3 * l], w[4 + 3 * l]
            M = self._agg(H)
            Z = H @ Ws + M @ Wn + b
            cache.append((H, M, Z))
            H = np.maximum(Z, 0.0)
        Y = H @ w[-2] + w[-1]
        cache.append(H)
        return (Y, cache) if keep else Y

    def loss_and_grads(self, params, X, Yt, scale, round_bf16=True):
        """Loss and gradients with respect to every parameter (FP32 masters;
        the bfloat16 rounding is treated as the identity, as a
        straight-through estimator)."""
        w = self._weights(params, round_bf16)
        Y, cache = self.forward(params, X, keep=True, round_bf16=round_bf16)
        R = Y.shape[0]
        c = np.asarray(scale, np.float64)
        diff = Y - np.asarray(Yt, np.float64)
        loss = float(np.sum(c * diff * diff) / R)
        dY = 2.0 * c * diff / R
        grads = [None] * len(params)
        H3 = cache[-1]
        grads[-2] = H3.T @ dY
        grads[-1] = dY.sum(axis=0)
        dH = dY @ w[-2].T
        for l in reversed(range(N_MP)):
            H, M, Z = cache[1 + l]
            Ws, Wn = w[2 + 3 * l], w[3 + 3 * l]
            dZ = dH * (Z > 0)
            grads[2 + 3 * l] = H.T @ dZ
            grads[3 + 3 * l] = M.T @ dZ
            grads[4 + 3 * l] = dZ.sum(axis=0)
            dH = dZ @ Ws.T + self._agg_t(dZ @ Wn.T)
        X, Z0 = cache[0]
        dZ0 = dH * (Z0 > 0)
        grads[0] = X.T @ dZ0
        grads[1] = dZ0.sum(axis=0)
        return loss, grads
