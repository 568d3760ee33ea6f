"""Learned warm start for the message-passing iteration (include/opf_wsnet.h).

The paper has no learned component; its warm start (Section 3.4) reuses a
previous solution.  Here a three-layer message-passing network over the bus
graph, trained on solutions of load-perturbed instances of one network,
proposes the nodal prices and base-case node angles of a new instance; they
set the starting state, and the iteration then runs unchanged to the same
tolerance.

Starting state from predicted prices lambda[n, t] and angles theta[n, t]
(``warm_state``): the prices are -rho_p sum_k u_k at a fixed point of step 2
(Section 3.2), so every contingency gets u_k = -lambda / (rho_p (K+1)) at the
context's initial rho_p; every line terminal takes its node's angle, the
line power is b (theta_1 - theta_2) clipped to the limit (0 on the outaged
line of a contingency), and v = 0 (so v_bar = 0 holds), device powers 0.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 9
PRICE_SCALE = 100.0


def node_features(case):
    """Features [T * N, 9] of every (step t, node n), rows t * N + n: load,
    generation capacity (max and min), cheapest linear generation cost,
    battery power, line count, summed susceptance, and the time of day."""
    N, T = int(case["n_nodes"]), int(case["T"])
    f = np.zeros((T, N, N_FEATURES))
    gn = np.asarray(case["gen_node"])
    np.add.at(f[:, :, 0], (slice(None), np.asarray(case["load_node"])), np.asarray(case["load_p"]).T)
    np.add.at(f[:, :, 1], (slice(None), gn), np.asarray(case["gen_pmax"]).T)
    np.add.at(f[:, :, 2], (slice(None), gn), np.asarray(case["gen_pmin"]).T)
    cheapest = np.zeros(N)
    has = np.zeros(N, bool)
    for g, b in zip(gn, case["gen_b"]):
        cheapest[g] = b if not has[g] else min(cheapest[g], b)
        has[g] = True
    f[:, :, 3] = cheapest[None, :] / PRICE_SCALE
    np.add.at(f[:, :, 4], (slice(None), np.asarray(case["stor_node"])), np.asarray(case["stor_P"])[None, :])
    deg = np.zeros(N)
    bs = np.zeros(N)
    for a, c, b in zip(case["line_from"], case["line_to"], case["line_b"]):
        deg[a] += 1
        deg[c] += 1
        bs[a] += b
        bs[c] += b
    f[:, :, 5] = deg[None, :]
    f[:, :, 6] = bs[None, :] / 100.0
    t = np.arange(T)[:, None]
    f[:, :, 7] = np.sin(2 * np.pi * t / 24.0)
    f[:, :, 8] = np.cos(2 * np.pi * t / 24.0)
    return f.reshape(T * N, N_FEATURES)


def targets(price, theta_base):
    """Targets [T * N, 2] from prices [N][T] and base-case angles [N][T]."""
    return np.stack([np.asarray(price).T.ravel() / PRICE_SCALE, np.asarray(theta_base).T.ravel()], axis=1)


def warm_state(case, y, rho_p=1.0):
    """The starting state (opf_state arrays) from network outputs y [T * N, 2]."""
    N, T = int(case["n_nodes"]), int(case["T"])
    out = np.asarray(case["outaged"])
    Kp = len(out) + 1
    lam = (y[:, 0] * PRICE_SCALE).reshape(T, N).T          # [N][T]
    th = y[:, 1].reshape(T, N).T
    lf, lt = np.asarray(case["line_from"]), np.asarray(case["line_to"])
    lb, lu = np.asarray(case["line_b"], float), np.asarray(case["line_u"], float)
    L = len(lf)
    t1, t2 = th[lf], th[lt]                                # [L][T]
    p = np.clip(lb[:, None] * (t1 - t2), -lu[:, None], lu[:, None])
    p_line = np.repeat(p[None], Kp, axis=0)
    for k, l in enumerate(out, start=1):
        if l >= 0:
            p_line[k, l] = 0.0
    S = (len(case["gen_node"]) + len(case["load_node"]) + len(case["stor_node"])
         + 2 * len(case.get("hvdc_from", ())))
    u = np.repeat((-lam / (rho_p * Kp))[None], Kp, axis=0)
    f32 = np.float32
    return dict(p_line=p_line.astype(f32), th1=np.repeat(t1[None], Kp, 0).astype(f32),
                th2=np.repeat(t2[None], Kp, 0).astype(f32), v1=np.zeros((Kp, L, T), f32),
                v2=np.zeros((Kp, L, T), f32), p_dev=np.zeros((S, T), f32), u=u.astype(f32))


class Normalizer:
    """Per-feature mean and spread of the training inputs."""

    def __init__(self, X):
        self.mean = X.mean(axis=0)
        self.std = np.where(X.std(axis=0) > 1e-9, X.std(axis=0), 1.0)

    def __call__(self, X):
        return ((X - self.mean) / self.std).astype(np.float32)


def train(net, xs, ys, epochs, lr, scale=(1.0, 1.0), seed=0, on_epoch=None):
    """Adam over the instances (one instance per step, shuffled each epoch);
    xs, ys are lists of device tensors.  Returns the mean loss per epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(xs))
        tot = 0.0
        for i in order:
            tot += net.train_step(xs[i], ys[i], scale, lr)
        hist.append(tot / len(xs))
        if on_epoch:
            on_epoch(ep, hist[-1])
    return hist
