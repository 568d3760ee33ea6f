"""Plain FP64 restatement of proximal message passing for contingency DC OPF.

TEST INFRASTRUCTURE ONLY -- imported by tests, the smoke check and the CPU
baseline of the benchmark; never by the product library.

The code follows the paper's notation (Appendix A): terminals ``j``, nodes
``n``, contingencies ``k = 0..K``; the state is ``s = (p, theta, u, v)``
(Section 4.4) with ``p`` kept per terminal, shape ``[K+1, J, T]``,
``theta, v`` per phase terminal (the ``2L`` line terminals), shape
``[K+1, 2L, T]``, and ``u`` per node, shape ``[K+1, N, T]`` (Section 4.1
stores node-constant quantities per node; ``u`` is node-constant because
``u~ = 0``, Section 3.2).

Terminal order: terminal 1 of every line, terminal 2 of every line, then
generators, loads and batteries (one terminal each).

Readings of passages where the paper is garbled or silent, each with the
reason it is taken:

* generator prox: ``clip((rho x - b) / (2 a + rho), pmin, pmax)`` -- Section
  4.2 prints the fraction upside down;
* line prox: the denominator is ``2 rho_p + rho_theta / (2 b^2)`` -- Section
  4.2 prints ``2 (rho_p + rho_theta + 1/4b^2)``; an outaged line (``u = b =
  0``, Section 2.3) decouples its terminals: ``p = 0, theta = y``;
* non-contingency prox input: ``p_d - avg_k(pbar_kd + u_kd)`` -- Section 3.2
  prints ``- u``; ``+ u`` is what eliminating ``z = p~`` gives and matches
  step 1's ``p~ - u``;
* phase terminals: only devices whose cost involves an angle (the lines)
  carry a phase.  Generators, loads and batteries ignore ``theta``; if their
  terminals carried a phase shared by all contingencies (Eq.
  contingency-dispatch fixes ``theta_{k l} = theta_{0 l}`` for those types),
  phase consistency would pin every node angle to one value across all
  contingencies, which no outage of a loaded line can satisfy.  So
  ``theta_bar`` and ``theta~`` range over line terminals, and ``|n|_theta``
  counts the line terminals of node ``n``;
* residual norms are taken over terminal-level vectors (node quantities
  repeat ``|n|`` times, non-contingency terminals once per contingency); the
  stopping threshold keeps Eq. (converge)'s ``eps sqrt(2 J T (K+1))`` with
  ``J`` counting every terminal;
* inner ADMM (Appendix D): equality rows are split like inequality rows with
  ``beta`` projected onto ``{0}``; the dual update uses the new ``alpha`` and
  ``beta``; ``omega = rho'`` (the device's outer penalty); 10 inner iterations;
  ``(beta, lambda)`` warm-start across outer iterations and ``lambda`` is
  rescaled by ``omega_old / omega_new`` when ``omega`` changes;
* a ramp limit binds consecutive steps only; storage steps are one period
  long (``s_{t+1} = s_t + eff c_t - delta_t``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.sparse import csr_matrix


@dataclass
class OracleOptions:
    """Algorithm parameters (Section 3.5 and Section 5.2 defaults)."""

    rho_p: float = 1.0        # penalty for power balance
    rho_theta: float = 1.0    # penalty for phase consistency
    eps: float = 1e-4         # absolute tolerance of Eq. (converge); <= 0 disables stopping
    mu: float = 2.0           # residual-ratio threshold of the adaptive penalty
    gamma: float = 1.1        # penalty scaling factor
    adapt_every: int = 10     # i_adapt (0 disables adaptation)
    inner_iters: int = 10     # inner ADMM iterations per iterative prox (Appendix D)
    check_every: int = 10     # stopping test cadence (0 = never)
    alpha: float = 1.0        # over-relaxation parameter in [1, 2) (Section 3.6); 1 = plain ADMM
    # Not in the paper (Section 3.5 adapts for the whole run): the residual
    # balancing rule it takes from Boyd et al. (2011, Section 3.4.1) keeps
    # ADMM's convergence guarantee only if the penalty stops changing after
    # finitely many iterations.
    adapt_until: int = 0      # last iteration that may adapt (0 = no limit)
    stall_window: int = 0     # progress window of the stopping test (0 = off); see Oracle._stall


# ---------------------------------------------------------------------------
# device proximal operators
# ---------------------------------------------------------------------------

def prox_gen(x, a, b, pmin, pmax, rho):
    """Prox of ``a p^2 + b p + I{pmin <= p <= pmax}`` with weight ``rho``.

    Section 2.1 (generator; curtailable load with ``pmin < pmax <= 0``) and
    Section 4.2 (analytical update).  Setting the derivative of
    ``a p^2 + b p + rho/2 (p - x)^2`` to zero gives ``(rho x - b)/(2a + rho)``;
    for a separable convex quadratic the box constraint is a clip.  The angle
    is free, so ``theta = y``.
    """
    return np.clip((rho * x - b) / (2.0 * a + rho), pmin, pmax)


def prox_fixed_load(x, P):
    """Prox of ``I{p = -P}`` (Section 2.1 fixed load, ``P`` consumed): ``p = -P``."""
    return np.broadcast_to(-np.asarray(P, float), np.shape(x)).copy()


def prox_line(x1, x2, y1, y2, u, b, rho_p, rho_theta, active):
    """Prox of the DC line cost ``f^ac`` (Section 2.1) with weights ``rho_p, rho_theta``.

    ``f^ac = I{p1 + p2 = 0} + I{|p2| <= u} + I{p2 = b (theta1 - theta2)}``.
    Eliminating ``p1 = -p2`` and minimising over ``theta1 + theta2`` at fixed
    ``theta1 - theta2 = p2 / b`` leaves a 1-D convex quadratic in ``p2``:
    ``rho_p/2 ((p2 + x1)^2 + (p2 - x2)^2) + rho_theta/4 (p2/b - (y1 - y2))^2``,
    minimised over ``[-u, u]`` by clipping the stationary point
    ``(rho_p (x2 - x1) + rho_theta (y1 - y2) / (2b)) / (2 rho_p + rho_theta / (2 b^2))``.
    Then ``theta1,2 = (y1 + y2)/2 +- p2 / (2b)``.  Where ``active`` is false
    (the outaged line of a contingency, ``u = b = 0``, Section 2.3) the
    terminals decouple: ``p1 = p2 = 0`` and ``theta = y``.

    Returns ``(p1, p2, theta1, theta2)``.
    """
    active = np.asarray(active, bool)
    bs = np.where(active, b, 1.0)
    num = rho_p * (x2 - x1) + rho_theta * (y1 - y2) / (2.0 * bs)
    den = 2.0 * rho_p + rho_theta / (2.0 * bs * bs)
    p2 = np.clip(num / den, -u, u)
    mid = 0.5 * (y1 + y2)
    th1 = mid + p2 / (2.0 * bs)
    th2 = mid - p2 / (2.0 * bs)
    p2 = np.where(active, p2, 0.0)
    th1 = np.where(active, th1, y1)
    th2 = np.where(active, th2, y2)
    return -p2, p2, th1, th2


# ---------------------------------------------------------------------------
# iterative proxes: Appendix D inner ADMM on f = min_s s'Qs + q's + I{A z <= h}
# ---------------------------------------------------------------------------

def prox_hvdc(x1, x2, u):
    """Prox of an HVDC link (Section 2.1, other devices): two terminals with
    ``p1 + p2 = 0`` and ``|p2| <= u`` and no angle relation (the link is
    converter-controlled).  Minimising ``(rho/2)((p1 - x1)^2 + (p2 - x2)^2)``
    over ``p1 = -p2`` is ``(rho/2)((p2 + x1)^2 + (p2 - x2)^2)``, a parabola
    with vertex ``(x2 - x1)/2``; the limit clips it.  Independent of rho.
    Returns ``(p1, p2)``."""
    p2 = np.clip((x2 - x1) / 2.0, -u, u)
    return -p2, p2


def ramp_rows(pmin, pmax, R):
    """Constraint rows ``A p <= h`` of a generator with box and ramp limits
(the ramp-limited generator of Section 2.1, in the ``A x <= h`` form of
Appendix D).

    Variables ``z = p`` (length T).  Rows: ``p_t <= pmax_t``,
    ``-p_t <= -pmin_t``, ``p_{t+1} - p_t <= R`` and ``p_t - p_{t+1} <= R``
    for consecutive steps.  Returns ``(A, h, eq)``; no equality rows.
    """
    pmin = np.asarray(pmin, float)
    pmax = np.asarray(pmax, float)
    T = len(pmin)
    I = np.eye(T)
    Dm = I[1:] - I[:-1]
    A = np.vstack([I, -I, Dm, -Dm])
    h = np.concatenate([pmax, -pmin, np.full(T - 1, R), np.full(T - 1, R)])
    return A, h, np.zeros(len(h), bool)


def storage_layout(T):
    """Index slices of ``z = (p, c, delta, s)`` for a battery with horizon T
    (the storage device of Section 2.1: power, charge, discharge, state of
    charge)."""
    return (slice(0, T), slice(T, 2 * T), slice(2 * T, 3 * T), slice(3 * T, 4 * T + 1))


def storage_rows(T, eff, P, dur):
    """Constraint rows of the battery cost ``f^store`` (Section 2.1).

    Variables ``z = (p, c, delta, s)`` with ``s`` of length ``T + 1``.
    Equality rows (``eq = True``): ``p_t + c_t - delta_t = 0`` (device power
    balance ``p = delta - c``), ``s_{t+1} - s_t - eff c_t + delta_t = 0``
    (state of charge), ``s_1 = 0`` and ``s_{T+1} = 0``.  Inequality rows:
    ``0 <= c <= P``, ``0 <= delta <= P``, ``0 <= s <= dur P``.
    Returns ``(A, h, eq)``.
    """
    sp, sc, sd, ss = storage_layout(T)
    n = 4 * T + 1
    rows, hs, eqs = [], [], []

    def row():
        r = np.zeros(n)
        rows.append(r)
        return r

    for t in range(T):                      # p_t + c_t - delta_t = 0
        r = row()
        r[sp.start + t] = 1.0
        r[sc.start + t] = 1.0
        r[sd.start + t] = -1.0
        hs.append(0.0)
        eqs.append(True)
    for t in range(T):                      # s_{t+1} - s_t - eff c_t + delta_t = 0
        r = row()
        r[ss.start + t + 1] = 1.0
        r[ss.start + t] = -1.0
        r[sc.start + t] = -eff
        r[sd.start + t] = 1.0
        hs.append(0.0)
        eqs.append(True)
    for idx in (ss.start, ss.start + T):    # s_1 = 0, s_{T+1} = 0
        r = row()
        r[idx] = 1.0
        hs.append(0.0)
        eqs.append(True)
    for sl, hi, cnt in ((sc, P, T), (sd, P, T), (ss, dur * P, T + 1)):
        for t in range(cnt):                # x <= hi
            r = row()
            r[sl.start + t] = 1.0
            hs.append(hi)
            eqs.append(False)
        for t in range(cnt):                # -x <= 0
            r = row()
            r[sl.start + t] = -1.0
            hs.append(0.0)
            eqs.append(False)
    return np.array(rows), np.array(hs), np.array(eqs, bool)


def inner_matrix(Qdiag, rho, omega, A, n_p):
    """System matrix of the Appendix D x-update, one per device.

    ``M = 2 diag(Q) + rho E_p + omega A'A`` where ``E_p`` selects the first
    ``n_p`` entries of ``z`` (the terminal power, which carries the prox term
    ``rho/2 ||p - x||^2``).  ``Qdiag``: ``[n_dev, n]``; returns ``[n_dev, n, n]``.
    """
    n = A.shape[1]
    Ep = np.zeros(n)
    Ep[:n_p] = 1.0
    base = omega * (A.T @ A)
    M = np.broadcast_to(base, (Qdiag.shape[0], n, n)).copy()
    idx = np.arange(n)
    M[:, idx, idx] += 2.0 * Qdiag + rho * Ep
    return M


def inner_admm(x, A, h, eq, q, rho, omega, Minv, beta, lam, n_iter):
    """``n_iter`` iterations of the Appendix D ADMM for a batch of devices.

    Minimises ``z'Qz + q'z + rho/2 ||z_p - x||^2 + I{A z <= h}`` via the split
    ``A z - h = alpha``, ``alpha = beta``, ``beta <= 0`` (``beta = 0`` on
    equality rows):

    1. ``z = M^{-1} (rho E_p' x - q + omega A'(h + beta - lam))`` -- the
       minimiser of the quadratic with ``alpha = A z - h`` substituted;
    2. ``alpha = A z - h``; ``beta = min(alpha + lam, 0)`` (``0`` on equality rows);
    3. ``lam = lam + alpha - beta``.

    Shapes: ``x [d, n_p]``, ``A [m, n]`` (shared), ``h [d, m]``, ``q [d, n]``,
    ``Minv [d, n, n]`` (cached inverse of ``inner_matrix``), ``beta, lam [d, m]``.
    Returns ``(z, beta, lam)`` with ``z`` from the last x-update.
    """
    n_p = x.shape[1]
    z = None
    for _ in range(n_iter):
        rhs = -q + omega * ((h + beta - lam) @ A)
        rhs[:, :n_p] += rho * x
        z = np.einsum("dij,dj->di", Minv, rhs)
        alpha = z @ A.T - h
        beta = np.where(eq, 0.0, np.minimum(alpha + lam, 0.0))
        lam = lam + alpha - beta
    return z, beta, lam


# ---------------------------------------------------------------------------
# network, averages and residuals (Eq. average-op, Eq. residual-op, Appendix B)
# ---------------------------------------------------------------------------

class Network:
    """Device-node model of an instance (Section 2, Section 2.2 type sets).

    Power terminals: every terminal (``J = 2L + G + D + B + 2H``, two per
    HVDC link, terminal 1 then 2 of each link).  Phase terminals: the ``2L``
    AC-line terminals (the first ``2L`` power terminals).  HVDC links are
    not of the contingency type (Section 2.3: only the first type, AC lines,
    changes per contingency), so like the other devices they keep one
    schedule for every contingency.
    """

    def __init__(self, case, k_ids=None):
        self.case = case
        self.T = int(case["T"])
        self.N = int(case["n_nodes"])
        lf = np.asarray(case["line_from"], np.int64)
        lt = np.asarray(case["line_to"], np.int64)
        self.line_from, self.line_to = lf, lt
        self.L = len(lf)
        self.gen_node = np.asarray(case["gen_node"], np.int64)
        self.load_node = np.asarray(case["load_node"], np.int64)
        self.stor_node = np.asarray(case["stor_node"], np.int64)
        self.G, self.D, self.B = len(self.gen_node), len(self.load_node), len(self.stor_node)
        self.outaged = np.asarray(case["outaged"], np.int64)
        self.K = len(self.outaged)
        # contingencies held here: all of 0..K, or a shard of them (k_ids)
        self.k_ids = np.arange(self.K + 1) if k_ids is None else np.asarray(k_ids, np.int64)
        self.Kp = len(self.k_ids)
        L, G, D, B = self.L, self.G, self.D, self.B
        self.sl_t1 = slice(0, L)
        self.sl_t2 = slice(L, 2 * L)
        self.sl_dev = slice(2 * L, 2 * L + G + D + B + 2 * len(case.get("hvdc_from", ())))
        hf = np.asarray(case.get("hvdc_from", ()), np.int64)
        ht = np.asarray(case.get("hvdc_to", ()), np.int64)
        self.H = len(hf)
        self.hvdc_u = np.asarray(case.get("hvdc_u", ()), float)
        hv = np.empty(2 * self.H, np.int64)
        hv[0::2], hv[1::2] = hf, ht
        self.term_node = np.concatenate([lf, lt, self.gen_node, self.load_node, self.stor_node, hv])
        self.J = len(self.term_node)
        self.S = G + D + B + 2 * self.H
        # node-terminal incidence (Appendix B: A = L' diag(|n|)^-1 L), for
        # power (all terminals) and for phase (line terminals)
        self.Linc = csr_matrix((np.ones(self.J), (self.term_node, np.arange(self.J))),
                               shape=(self.N, self.J))
        self.count = np.asarray(self.Linc.sum(axis=1)).ravel()
        if np.any(self.count == 0):
            raise ValueError("every node needs at least one terminal")
        ph = self.term_node[:2 * L]
        self.Linc_th = csr_matrix((np.ones(2 * L), (ph, np.arange(2 * L))), shape=(self.N, 2 * L))
        self.count_th = np.asarray(self.Linc_th.sum(axis=1)).ravel()
        # contingency k: line outaged[k-1] has u = b = 0 (Section 2.3, N-1
        # example); an index of -1 keeps the base-case parameters
        self.active = np.ones((self.Kp, L), bool)
        for i, k in enumerate(self.k_ids):
            if k > 0 and self.outaged[k - 1] >= 0:
                self.active[i, self.outaged[k - 1]] = False
        self.line_b = np.asarray(case["line_b"], float)
        self.line_u = np.asarray(case["line_u"], float)
        self.gen_a = np.asarray(case["gen_a"], float)
        self.gen_b = np.asarray(case["gen_b"], float)
        self.gen_pmin = np.asarray(case["gen_pmin"], float).reshape(G, self.T)
        self.gen_pmax = np.asarray(case["gen_pmax"], float).reshape(G, self.T)
        self.gen_ramp = np.asarray(case["gen_ramp"], float)
        self.is_ramp = (self.gen_ramp >= 0) & (self.T > 1)
        self.load_p = np.asarray(case["load_p"], float).reshape(D, self.T)
        self.load_voll = np.asarray(case["load_voll"], float)
        self.is_fixed = self.load_voll < 0
        self.stor_P = np.asarray(case["stor_P"], float)
        self.stor_dur = np.asarray(case["stor_dur"], float)
        self.stor_eff = np.asarray(case["stor_eff"], float)
        self.stor_cost = np.asarray(case["stor_cost"], float)


def node_mean(net, z, phase=False):
    """Node averages ``(1/|n|) sum_{j in n} z_j`` -> ``[K+1, N, T]``.

    Eq. (average-op), computed as ``diag(|n|)^-1 L z`` with the node-terminal
    incidence ``L`` (Section 4.3 / Appendix B).  ``z`` is ``[K+1, J, T]`` over
    power terminals, or with ``phase`` ``[K+1, 2L, T]`` over phase terminals;
    a node without phase terminals gets 0.
    """
    Linc, cnt = (net.Linc_th, net.count_th) if phase else (net.Linc, net.count)
    safe = np.where(cnt > 0, cnt, 1.0)
    out = np.empty((z.shape[0], net.N, z.shape[2]))
    for k in range(z.shape[0]):
        out[k] = (Linc @ z[k]) / safe[:, None]
    return out


def average(net, z, phase=False):
    """Terminal-level average ``z_bar_j`` (Eq. average-op), shape of ``z``."""
    idx = net.term_node[:2 * net.L] if phase else net.term_node
    return node_mean(net, z, phase)[:, idx, :]


def residual(net, z, phase=False):
    """Terminal-level residual ``z~ = z - z_bar`` (Eq. residual-op)."""
    return z - average(net, z, phase)


# ---------------------------------------------------------------------------
# the iteration
# ---------------------------------------------------------------------------

class Shard:
    """A slice of the contingencies for one of several cooperating processes.

    ``k_ids`` are the global contingency indices held locally and
    ``allreduce(x)`` returns the elementwise sum of ``x`` over all processes.
    The only quantities that couple contingencies are the sums over ``k``
    feeding the non-contingency proxes (Section 3.2) and the residual norms
    (Section 3.3), so those are the two places that call it.
    """

    def __init__(self, k_ids, K, allreduce):
        self.k_ids = np.asarray(k_ids, np.int64)
        self.Kp_total = K + 1
        self.allreduce = allreduce


class Oracle:
    """Proximal message passing (Section 3.2) with residuals (Section 3.3) and
    the adaptive penalty (Section 3.5), over all contingencies and time steps
    (or over a ``Shard`` of the contingencies)."""

    def __init__(self, case, opts=None, shard=None):
        self.shard = shard
        self.net = Network(case, None if shard is None else shard.k_ids)
        self.Kp_total = self.net.Kp if shard is None else shard.Kp_total
        self.opts = opts or OracleOptions()
        net = self.net
        Kp, J, N, T, L = net.Kp, net.J, net.N, net.T, net.L
        self.p = np.zeros((Kp, J, T))
        self.th = np.zeros((Kp, 2 * L, T))
        self.v = np.zeros((Kp, 2 * L, T))
        self.u = np.zeros((Kp, N, T))
        # duplicate variables of the over-relaxed form (Section 3.6)
        self.z = np.zeros((Kp, J, T))
        self.xi = np.zeros((Kp, 2 * L, T))
        self.rho_p = float(self.opts.rho_p)
        self.rho_th = float(self.opts.rho_theta)
        self.it = 0
        self.res = np.zeros(6)
        self.converged = False
        self.rho_history = []
        # the stall rule's state (Oracle._stall)
        self.frozen_at = 0        # iteration at which the rule fixed the penalties (0 = never)
        self.stalled = False
        self.stall_ref = np.inf   # best max(||r_primal||, ||r_dual||) at a stopping test ...
        self.stall_it = 0         # ... and the iteration where it was reached
        self._conv_now = False    # the last iteration passed a stopping test
        # inner ADMM state of the iterative proxes
        self.ramp_idx = np.nonzero(net.is_ramp)[0]
        if len(self.ramp_idx):
            A, _, _ = ramp_rows(np.zeros(T), np.zeros(T), 0.0)
            self.ramp_A = A
            self.ramp_eq = np.zeros(A.shape[0], bool)
            self.ramp_h = np.stack([ramp_rows(net.gen_pmin[g], net.gen_pmax[g],
                                              net.gen_ramp[g])[1] for g in self.ramp_idx])
            m = A.shape[0]
            self.ramp_beta = np.zeros((len(self.ramp_idx), m))
            self.ramp_lam = np.zeros((len(self.ramp_idx), m))
        if net.B:
            self.stor_groups = {}
            for b in range(net.B):
                self.stor_groups.setdefault(float(net.stor_eff[b]), []).append(b)
            self.stor_A, self.stor_eq = {}, {}
            for eff in self.stor_groups:
                A, _, eq = storage_rows(T, eff, 0.0, 0.0)
                self.stor_A[eff], self.stor_eq[eff] = A, eq
            self.stor_h = np.stack([storage_rows(T, net.stor_eff[b], net.stor_P[b],
                                                 net.stor_dur[b])[1] for b in range(net.B)])
            m = self.stor_h.shape[1]
            self.stor_beta = np.zeros((net.B, m))
            self.stor_lam = np.zeros((net.B, m))
            self.stor_z = np.zeros((net.B, 4 * T + 1))
        self._factored_rho = None

    # -- cached inner factorizations (Appendix D: reused while rho, omega fixed)
    def _factor(self):
        """Inverse x-update matrices of the inner ADMM (Appendix D) at the
        current device weight (K+1) rho_p, recomputed when it changes."""
        rho = self.Kp_total * self.rho_p
        if self._factored_rho == rho:
            return
        net, T = self.net, self.net.T
        omega = rho
        if len(self.ramp_idx):
            Qd = np.repeat(net.gen_a[self.ramp_idx][:, None], T, axis=1)
            self.ramp_Minv = np.linalg.inv(inner_matrix(Qd, rho, omega, self.ramp_A, T))
        if net.B:
            self.stor_Minv = np.empty((net.B, 4 * T + 1, 4 * T + 1))
            for eff, members in self.stor_groups.items():
                Qd = np.zeros((len(members), 4 * T + 1))
                self.stor_Minv[members] = np.linalg.inv(
                    inner_matrix(Qd, rho, omega, self.stor_A[eff], T))
        self._factored_rho = rho

    # -- state import (the C ABI's export layout: include/opf.h opf_state)
    def load_state(self, st, rho_p=None, rho_theta=None, it=None):
        """Set the iterate from a state dict with keys p_line, th1, th2, v1, v2
        ``[K+1, L, T]``, p_dev ``[S, T]``, u ``[K+1, N, T]`` and optionally
        ``inner`` (ramp generators then batteries, each lambda then beta over
        the rows of ``ramp_rows`` / ``storage_rows``): the warm start of
        Section 3.4, which restarts the iteration from a given state."""
        net = self.net
        L = net.L
        f = lambda x: np.asarray(x, dtype=np.float64)
        self.p[:, :L] = -f(st["p_line"])
        self.p[:, L:2 * L] = f(st["p_line"])
        self.p[:, net.sl_dev] = f(st["p_dev"])[None]
        self.th[:, :L] = f(st["th1"])
        self.th[:, L:] = f(st["th2"])
        self.v[:, :L] = f(st["v1"])
        self.v[:, L:] = f(st["v2"])
        self.u[:] = f(st["u"])
        # the over-relaxed form restarts its duplicates where plain ADMM has
        # them: z = p~, xi = theta_bar
        self.z = self.p - average(net, self.p)
        self.xi = average(net, self.th, phase=True)
        if rho_p is not None:
            self.rho_p = float(rho_p)
        if rho_theta is not None:
            self.rho_th = float(rho_theta)
        if it is not None:
            self.it = int(it)
        # a warm start restarts the stall rule with adapting penalties
        self.frozen_at, self.stalled = 0, False
        self.stall_ref, self.stall_it = np.inf, self.it
        inner = st.get("inner")
        if inner is not None:
            x = f(inner)
            o = 0
            if len(self.ramp_idx):
                m = self.ramp_A.shape[0]
                for r in range(len(self.ramp_idx)):
                    self.ramp_lam[r] = x[o:o + m]
                    self.ramp_beta[r] = x[o + m:o + 2 * m]
                    o += 2 * m
            if net.B:
                m = self.stor_h.shape[1]
                for b in range(net.B):
                    self.stor_lam[b] = x[o:o + m]
                    self.stor_beta[b] = x[o + m:o + 2 * m]
                    o += 2 * m
            assert o == len(x)

    # -- state access
    def line_p(self):
        """Terminal-2 power of every line, ``[K+1, L, T]``."""
        return self.p[:, self.net.sl_t2]

    def dev_p(self):
        """Power of the non-contingency devices (gens, loads, batteries), ``[S, T]``."""
        return self.p[0, self.net.sl_dev]

    def pbar(self):
        """Node means of terminal power, ``[K+1, N, T]`` (Eq. average-op)."""
        return node_mean(self.net, self.p)

    def thbar(self):
        """Node means of line-terminal angles, ``[K+1, N, T]`` (Eq. average-op)."""
        return node_mean(self.net, self.th, phase=True)

    def prices(self):
        """Nodal prices ``-rho_p sum_k u_k`` (stationarity of step 2 at a fixed point)."""
        s = self.u.sum(axis=0)
        if self.shard is not None:
            s = self.shard.allreduce(s)
        return -self.rho_p * s

    def objective(self):
        """Sum of device costs at the current iterate, the objective of Eq.
        contingency-dispatch (line costs are indicators)."""
        net = self.net
        pd = self.dev_p()
        pg = pd[:net.G]
        f = float(np.sum(net.gen_a[:, None] * pg * pg + net.gen_b[:, None] * pg))
        pl = pd[net.G:net.G + net.D]
        cur = ~net.is_fixed
        f += float(np.sum(net.load_voll[cur, None] * (pl[cur] + net.load_p[cur])))
        if net.B:
            _, _, sdl, _ = storage_layout(net.T)
            f += float(np.sum(net.stor_cost[:, None] * self.stor_z[:, sdl]))
        return f

    # -- one iteration
    def step(self):
        """One message-passing iteration (Section 3.2): step 1 the line proxes
        of every contingency, step 2 the shared devices' proxes, step 3 the
        node averages and scaled price updates, then the residuals of Section
        3.3 and the adaptive penalty of Section 3.5."""
        if self.opts.alpha != 1.0:
            return self._step_relaxed()
        net = self.net
        rp, rt = self.rho_p, self.rho_th
        p, th, u, v = self.p, self.th, self.u, self.v
        tn = net.term_node

        pbar = average(net, p)
        thbar = average(net, th, phase=True)
        uj = u[:, tn, :]
        ptil_old = p - pbar
        thbar_old = thbar

        # step 1 at prox(p~ - u, theta_bar - v); step 2 at p_d - avg_k(pbar_kd + u_kd)
        sd = net.sl_dev
        p_new, th_new = self._proxes(ptil_old - uj, thbar - v,
                                     p[0, sd] - self._kmean(pbar[:, sd] + uj[:, sd]))

        # step 3: scaled price updates u += pbar, v += theta~
        pbar_new_n = node_mean(net, p_new)
        pbar_new = pbar_new_n[:, tn, :]
        thbar_new = average(net, th_new, phase=True)
        u_new = u + pbar_new_n
        v_new = v + (th_new - thbar_new)

        # residuals (Section 3.3), with the penalties used in this iteration
        r_pp = self._norm(pbar_new)
        r_pt = self._norm(th_new - thbar_new)
        r_dp = rp * self._norm((p_new - pbar_new) - ptil_old)
        r_dt = rt * self._norm(thbar_new - thbar_old)
        self._finish(p_new, th_new, u_new, v_new, r_pp, r_pt, r_dp, r_dt)

    def _finish(self, p_new, th_new, u_new, v_new, r_pp, r_pt, r_dp, r_dt):
        """Store the new iterate and its residual parts (Section 3.3); on
        stopping-test iterations the test of Eq. (converge) and the stall
        rule; adapt the penalties on adaptation iterations (Section 3.5)."""
        self.res = np.array([np.hypot(r_pp, r_pt), np.hypot(r_dp, r_dt), r_pp, r_pt, r_dp, r_dt])
        self.p, self.th, self.u, self.v = p_new, th_new, u_new, v_new
        self.it += 1
        o = self.opts
        self._conv_now = False
        if o.eps > 0 and o.check_every and self.it % o.check_every == 0:
            self._conv_now = max(self.res[0], self.res[1]) <= self.tolerance()
            if not self._conv_now and o.stall_window > 0:
                self._stall()
        # adaptive penalty (Section 3.5), every adapt_every iterations
        if self._adapting() and self.it % o.adapt_every == 0:
            self._adapt(r_pp, r_pt, r_dp, r_dt)

    def _adapting(self):
        """Whether the penalties may still adapt at the current iteration."""
        o = self.opts
        return bool(o.adapt_every) and (o.adapt_until <= 0 or self.it <= o.adapt_until) and not self.frozen_at

    def _stall(self):
        """Stall rule at a stopping test that failed (not in the paper).  Let
        m = max(||r_primal||, ||r_dual||).  When m falls below 0.99 times the
        best value so far, that value and its iteration are recorded.  When
        no such fall has happened for stall_window iterations:

        * while the penalties still adapt, they are fixed from this iteration
          on (ADMM with a penalty that stops changing converges for a
          feasible convex problem; Boyd et al. 2011, Section 3.4.1) and the
          window restarts;
        * with fixed penalties the run is stalled: iteration stops (an
          infeasible problem keeps a primal residual bounded away from zero).
        """
        o = self.opts
        m = max(self.res[0], self.res[1])
        if m < 0.99 * self.stall_ref:
            self.stall_ref, self.stall_it = m, self.it
        elif self.it - self.stall_it >= o.stall_window:
            if self._adapting():
                self.frozen_at = self.it
                self.stall_ref, self.stall_it = m, self.it
            else:
                self.stalled = True

    def _step_relaxed(self):
        """One over-relaxed ADMM iteration (Section 3.6) in the original form
        of Section 3.1 with explicit duplicate variables z (every terminal)
        and xi (phase terminals):

        1-2. the proxes at (z - u, xi - v), and for the devices shared by all
             contingencies at avg_k(z_kd - u_kd) with weight (K+1) rho_p;
        3.   p^half = alpha p + (1 - alpha) z, theta^half likewise with xi;
             z = projection of p^half + u onto {zbar = 0} (the residual
             operator), xi = projection of theta^half + v onto {xi~ = 0}
             (the average operator);
        4.   u += p^half - z, v += theta^half - xi.
        Residuals: r = (p - z, theta - xi), s = (rho_p (z - z_prev),
        rho_theta (xi - xi_prev)).  With alpha = 1 this is the message
        passing step above."""
        net = self.net
        tn = net.term_node
        a, rp, rt = self.opts.alpha, self.rho_p, self.rho_th
        z, xi = self.z, self.xi
        uj = self.u[:, tn, :]
        sd = net.sl_dev
        p_new, th_new = self._proxes(z - uj, xi - self.v, self._kmean(z[:, sd] - uj[:, sd]))
        p_half = a * p_new + (1.0 - a) * z
        th_half = a * th_new + (1.0 - a) * xi
        w = p_half + uj
        u_node = node_mean(net, w)                      # average of p^half + u at each node
        z_new = w - u_node[:, tn, :]                    # residual operator: zbar = 0
        xi_new = average(net, th_half + self.v, phase=True)
        u_new = u_node                                  # u + p^half - z (node-constant)
        v_new = self.v + th_half - xi_new
        r_pp = self._norm(p_new - z_new)
        r_pt = self._norm(th_new - xi_new)
        r_dp = rp * self._norm(z_new - z)
        r_dt = rt * self._norm(xi_new - xi)
        self.z, self.xi = z_new, xi_new
        self._finish(p_new, th_new, u_new, v_new, r_pp, r_pt, r_dp, r_dt)

    def _proxes(self, x, y, X):
        """Steps 1 and 2: the line proxes of every contingency at (x, y)
        (terminal-level) and the shared devices at X [S][T]; returns the new
        terminal powers [Kp][J][T] and line angles [Kp][2L][T]."""
        net, o = self.net, self.opts
        Kp, T, L = net.Kp, net.T, net.L
        rp, rt = self.rho_p, self.rho_th
        p_new = np.empty((Kp, net.J, T))
        act = np.broadcast_to(net.active[:, :, None], (Kp, L, T))
        u_k = net.line_u[None, :, None] * act
        b_k = net.line_b[None, :, None] * act
        p1, p2, th1, th2 = prox_line(x[:, :L], x[:, L:2 * L], y[:, :L], y[:, L:],
                                     u_k, b_k, rp, rt, act)
        p_new[:, net.sl_t1], p_new[:, net.sl_t2] = p1, p2
        th_new = np.concatenate([th1, th2], axis=1)

        # step 2: non-contingency devices, one schedule shared by all k, prox
        # with weight (K+1) rho_p
        sd = net.sl_dev
        rho_d = self.Kp_total * rp
        self._factor()
        pd = np.empty_like(X)
        G, D, B = net.G, net.D, net.B
        # generators: closed form, or the inner ADMM when ramp limits couple steps
        Xg = X[:G]
        pg = prox_gen(Xg, net.gen_a[:, None], net.gen_b[:, None], net.gen_pmin, net.gen_pmax, rho_d)
        if len(self.ramp_idx):
            ri = self.ramp_idx
            q = np.repeat(net.gen_b[ri][:, None], T, axis=1)
            z, self.ramp_beta, self.ramp_lam = inner_admm(
                Xg[ri], self.ramp_A, self.ramp_h, self.ramp_eq, q, rho_d, rho_d,
                self.ramp_Minv, self.ramp_beta, self.ramp_lam, o.inner_iters)
            pg[ri] = z[:, :T]
        pd[:G] = pg
        # loads: fixed (I{p = -P}) or curtailable (generator with a = 0, b = voll, [-P, 0])
        Xl = X[G:G + D]
        pl = prox_gen(Xl, 0.0, net.load_voll[:, None], -net.load_p, 0.0, rho_d)
        pl[net.is_fixed] = prox_fixed_load(Xl[net.is_fixed], net.load_p[net.is_fixed])
        pd[G:G + D] = pl
        # batteries: iterative prox
        if B:
            _, _, sdl, _ = storage_layout(T)
            Xb = X[G + D:G + D + B]
            pb = np.empty_like(Xb)
            for eff, members in self.stor_groups.items():
                mb = np.asarray(members)
                q = np.zeros((len(mb), 4 * T + 1))
                q[:, sdl] = net.stor_cost[mb][:, None]
                z, bet, lam = inner_admm(
                    Xb[mb], self.stor_A[eff], self.stor_h[mb], self.stor_eq[eff], q,
                    rho_d, rho_d, self.stor_Minv[mb], self.stor_beta[mb], self.stor_lam[mb],
                    o.inner_iters)
                self.stor_beta[mb], self.stor_lam[mb], self.stor_z[mb] = bet, lam, z
                pb[mb] = z[:, :T]
            pd[G + D:G + D + B] = pb
        # HVDC links: closed form, one schedule for every contingency
        if net.H:
            h0, h1 = G + D + B, G + D + B + 2 * net.H
            pd[h0:h1:2], pd[h0 + 1:h1:2] = prox_hvdc(X[h0:h1:2], X[h0 + 1:h1:2], net.hvdc_u[:, None])
        p_new[:, sd] = pd[None]
        return p_new, th_new

    # -- the two couplings across contingencies (reduced over a shard's peers)
    def _kmean(self, a):
        """``(1/(K+1)) sum_k a_k`` over all contingencies (the average over k
        that step 2 of Section 3.2 takes for the shared devices)."""
        if self.shard is None:
            return np.mean(a, axis=0)
        return self.shard.allreduce(np.sum(a, axis=0)) / self.Kp_total

    def _norm(self, x):
        """Euclidean norm over all contingencies (the residual norms of
        Section 3.3)."""
        if self.shard is None:
            return np.linalg.norm(x)
        return float(np.sqrt(self.shard.allreduce(np.array([np.sum(x * x)]))[0]))

    def _adapt(self, r_pp, r_pt, r_dp, r_dt):
        """Residual balancing (Section 3.5): each penalty grows by gamma when
        its primal part exceeds mu times its dual part, shrinks by gamma in
        the opposite case; the scaled duals are rescaled by rho_old /
        rho_new so that the unscaled duals stay fixed."""
        o = self.opts

        def rule(rho, rprim, rdual):
            if rprim > o.mu * rdual:
                return rho * o.gamma
            if rdual > o.mu * rprim:
                return rho / o.gamma
            return rho

        new_p = rule(self.rho_p, r_pp, r_dp)
        new_t = rule(self.rho_th, r_pt, r_dt)
        self.rho_history.append((self.it, new_p, new_t))
        if new_p != self.rho_p:
            scale = self.rho_p / new_p
            self.u *= scale
            # omega = (K+1) rho_p: keep the unscaled inner duals omega * lam fixed
            if len(self.ramp_idx):
                self.ramp_lam *= scale
            if self.net.B:
                self.stor_lam *= scale
            self.rho_p = new_p
        if new_t != self.rho_th:
            self.v *= self.rho_th / new_t
            self.rho_th = new_t

    def tolerance(self):
        """Right-hand side of Eq. (converge): ``eps sqrt(2 J T (K+1))``."""
        n = self.net
        return self.opts.eps * np.sqrt(2.0 * n.J * n.T * self.Kp_total)

    def iterate(self, n_iters, stop=True):
        """Run up to ``n_iters`` iterations; with ``stop`` the run ends at the
        first stopping test (every ``check_every`` iterations) that passes
        Eq. (converge), or at a stall (``_stall``).  A stalled run restarts
        its stall window here.  Returns iterations run."""
        if self.stalled:
            self.stalled = False
            self.stall_ref, self.stall_it = np.inf, self.it
        done = 0
        for _ in range(n_iters):
            self.step()
            done += 1
            if stop and self._conv_now:
                self.converged = True
                break
            if stop and self.stalled:
                break
        return done
