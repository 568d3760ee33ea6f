"""Pins for the oracle's operators and one message-passing iteration (CPU only).

* Appendix B identities of the average and residual operators on random
  incidence;
* the message-passing form (Section 3.2, simplified) against the full ADMM
  updates 1-4 of Section 3.2 with explicit copies ``z, xi`` and per-terminal
  duals -- this pins the simplification, including the sign of ``u`` in the
  non-contingency prox input;
* the residuals of Section 3.3 recomputed with the dense average matrix
  ``A = L' diag(|n|)^-1 L`` of Appendix B;
* the invariant ``v_bar = 0`` (Section 3.2, Appendix C);
* the over-relaxed iteration (Section 3.6) against the same dense full ADMM
  with ``alpha p + (1 - alpha) z`` in the copy and price updates.
"""
import numpy as np
import pytest

from gridgen import make_case, scale_case
from oracle import Oracle, OracleOptions, average, node_mean, prox_gen, prox_fixed_load, prox_line
from oracle.mp import Network


def dense_average(term_node, n_nodes):
    """Appendix B: A = L' diag(|n|)^-1 L as a dense terminal x terminal matrix."""
    J = len(term_node)
    Lm = np.zeros((n_nodes, J))
    Lm[term_node, np.arange(J)] = 1.0
    cnt = Lm.sum(axis=1)
    inv = np.where(cnt > 0, 1.0 / np.where(cnt > 0, cnt, 1.0), 0.0)
    return Lm.T @ np.diag(inv) @ Lm


def small_case(**kw):
    cfg = scale_case(12, 3, 3, seed=5, ramp=False, stor_per_node=0.0, fixed_frac=0.5)
    cfg.update(kw)
    return make_case(cfg)


# --------------------------------------------------------------------------
# Appendix B
# --------------------------------------------------------------------------

def test_average_residual_identities(rng):
    case = make_case(scale_case(15, 4, 2, seed=3))
    net = Network(case)
    z = rng.normal(size=(net.Kp, net.J, net.T))
    avg = lambda w: average(net, w)
    res = lambda w: w - average(net, w)
    np.testing.assert_allclose(avg(avg(z)), avg(z), atol=1e-12)          # idempotent
    np.testing.assert_allclose(res(res(z)), res(z), atol=1e-12)
    np.testing.assert_allclose(avg(res(z)), 0.0, atol=1e-12)             # cancel each other
    np.testing.assert_allclose(res(avg(z)), 0.0, atol=1e-12)
    w = rng.normal(size=z.shape)
    assert abs(np.sum(avg(z) * w) - np.sum(z * avg(w))) < 1e-9          # symmetric
    A = dense_average(net.term_node, net.N)
    np.testing.assert_allclose(np.einsum("ij,kjt->kit", A, z), avg(z), atol=1e-12)
    # the phase average runs over line terminals only
    zt = rng.normal(size=(net.Kp, 2 * net.L, net.T))
    At = dense_average(net.term_node[:2 * net.L], net.N)
    np.testing.assert_allclose(np.einsum("ij,kjt->kit", At, zt), average(net, zt, phase=True),
                               atol=1e-12)


# --------------------------------------------------------------------------
# full ADMM (Section 3.2, updates 1-4) vs message passing
# --------------------------------------------------------------------------

class FullADMM:
    """Section 3.2 ADMM with explicit copies z, xi and duals u, v per terminal.

    Closed-form devices only (lines, generators without ramps, loads)."""

    def __init__(self, case, rho_p, rho_t, alpha=1.0):
        self.alpha = alpha
        self.net = net = Network(case)
        assert not net.is_ramp.any() and net.B == 0
        Kp, J, L, T = net.Kp, net.J, net.L, net.T
        self.rp, self.rt = rho_p, rho_t
        self.p = np.zeros((Kp, J, T))
        self.th = np.zeros((Kp, 2 * L, T))
        self.z = np.zeros((Kp, J, T))
        self.xi = np.zeros((Kp, 2 * L, T))
        self.u = np.zeros((Kp, J, T))
        self.v = np.zeros((Kp, 2 * L, T))
        self.Ap = dense_average(net.term_node, net.N)
        self.At = dense_average(net.term_node[:2 * L], net.N)

    def step(self):
        net, L, Kp = self.net, self.net.L, self.net.Kp
        # 1. contingency schedule: argmin g + rho/2 ||p - z + u||^2 + rho/2 ||th - xi + v||^2
        x = self.z - self.u
        y = self.xi - self.v
        act = np.broadcast_to(net.active[:, :, None], (Kp, L, net.T))
        p1, p2, t1, t2 = prox_line(x[:, :L], x[:, L:2 * L], y[:, :L], y[:, L:], net.line_u[None, :, None] * act,
                                   net.line_b[None, :, None] * act, self.rp, self.rt, act)
        p = np.empty_like(self.p)
        p[:, :L], p[:, L:2 * L] = p1, p2
        th = np.concatenate([t1, t2], axis=1)
        # 2. non-contingency schedule: argmin g + sum_k rho/2 ||p - z_k + u_k||^2
        sd = net.sl_dev
        X = np.mean(self.z[:, sd] - self.u[:, sd], axis=0)
        rho = Kp * self.rp
        G, D = net.G, net.D
        pd = np.empty_like(X)
        pd[:G] = prox_gen(X[:G], net.gen_a[:, None], net.gen_b[:, None], net.gen_pmin, net.gen_pmax, rho)
        pl = prox_gen(X[G:G + D], 0.0, net.load_voll[:, None], -net.load_p, 0.0, rho)
        pl[net.is_fixed] = prox_fixed_load(pl[net.is_fixed], net.load_p[net.is_fixed])
        pd[G:G + D] = pl
        p[:, sd] = pd[None]
        # over-relaxation (Section 3.6): the copies and prices see
        # alpha p + (1 - alpha) z in place of p (alpha = 1: plain ADMM)
        a = self.alpha
        ph = a * p + (1 - a) * self.z
        thh = a * th + (1 - a) * self.xi
        # 3. copies: projections onto {z_bar = 0} and {xi~ = 0}
        w = ph + self.u
        z = w - np.einsum("ij,kjt->kit", self.Ap, w)
        xi = np.einsum("ij,kjt->kit", self.At, thh + self.v)
        # 4. scaled prices
        self.u = self.u + ph - z
        self.v = self.v + thh - xi
        self.res = np.array([np.linalg.norm(p - z), np.linalg.norm(th - xi),
                             self.rp * np.linalg.norm(z - self.z), self.rt * np.linalg.norm(xi - self.xi)])
        self.p, self.th, self.z, self.xi = p, th, z, xi


@pytest.mark.parametrize("K", [0, 3])
def test_message_passing_equals_full_admm(K):
    case = small_case(K=K)
    ora = Oracle(case, OracleOptions(adapt_every=0, rho_p=1.3, rho_theta=7.0))
    ref = FullADMM(case, 1.3, 7.0)
    net = ora.net
    for _ in range(25):
        ora.step()
        ref.step()
        np.testing.assert_allclose(ora.p, ref.p, atol=1e-11)
        np.testing.assert_allclose(ora.th, ref.th, atol=1e-11)
        np.testing.assert_allclose(ora.u[:, net.term_node], ref.u, atol=1e-11)   # u~ = 0 kept
        np.testing.assert_allclose(ora.v, ref.v, atol=1e-11)


@pytest.mark.parametrize("K", [0, 3])
def test_over_relaxed_oracle_equals_full_admm(K):
    """Section 3.6 with alpha = 1.5: the oracle's explicit-copy step (node
    averages by CSR) against the dense full ADMM above, iterates, copies and
    the four residual parts."""
    case = small_case(K=K)
    ora = Oracle(case, OracleOptions(adapt_every=0, rho_p=1.3, rho_theta=7.0, alpha=1.5))
    ref = FullADMM(case, 1.3, 7.0, alpha=1.5)
    net = ora.net
    for _ in range(25):
        ora.step()
        ref.step()
        np.testing.assert_allclose(ora.p, ref.p, atol=1e-11)
        np.testing.assert_allclose(ora.th, ref.th, atol=1e-11)
        np.testing.assert_allclose(ora.z, ref.z, atol=1e-11)
        np.testing.assert_allclose(ora.xi, ref.xi, atol=1e-11)
        np.testing.assert_allclose(ora.u[:, net.term_node], ref.u, atol=1e-11)   # u stays node-constant
        np.testing.assert_allclose(ora.v, ref.v, atol=1e-11)
        np.testing.assert_allclose(ora.res[2:], ref.res, rtol=1e-10, atol=1e-12)
        # the invariants the simplification of Section 3.2 rests on also hold here
        np.testing.assert_allclose(node_mean(net, ora.z), 0.0, atol=1e-11)
        np.testing.assert_allclose(average(net, ora.v, phase=True), 0.0, atol=1e-11)


def test_sign_of_u_in_device_prox_matters():
    """Flipping the sign of u in the non-contingency input (as printed in
    Section 3.2) departs from the full ADMM -- the pin above would catch it."""
    case = small_case(K=2)
    ref = FullADMM(case, 1.0, 5.0)
    ora = Oracle(case, OracleOptions(adapt_every=0, rho_p=1.0, rho_theta=5.0))
    net = ora.net
    for _ in range(6):
        ref.step()
        ora.step()
    # recompute the device input with -u from the oracle's pre-step state
    pbar = average(net, ora.p)
    uj = ora.u[:, net.term_node]
    sd = net.sl_dev
    x_plus = ora.p[0, sd] - np.mean(pbar[:, sd] + uj[:, sd], axis=0)
    x_minus = ora.p[0, sd] - np.mean(pbar[:, sd] - uj[:, sd], axis=0)
    x_ref = np.mean(ref.z[:, sd] - ref.u[:, sd], axis=0)
    np.testing.assert_allclose(x_plus, x_ref, atol=1e-11)
    assert np.max(np.abs(x_minus - x_ref)) > 1e-3


# --------------------------------------------------------------------------
# residuals (Section 3.3) and invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("cfg", ["mixed", "tiny"])
def test_residuals_match_dense_definition(cfg):
    case = make_case(scale_case(14, 4, 2, seed=11)) if cfg == "mixed" else make_case("tiny")
    ora = Oracle(case, OracleOptions(adapt_every=0, rho_p=0.7, rho_theta=3.0))
    net = ora.net
    Ap = dense_average(net.term_node, net.N)
    At = dense_average(net.term_node[:2 * net.L], net.N)
    mul = lambda M, z: np.einsum("ij,kjt->kit", M, z)
    for _ in range(12):
        p0, th0 = ora.p.copy(), ora.th.copy()
        ora.step()
        p1, th1 = ora.p, ora.th
        r_pp = np.linalg.norm(mul(Ap, p1))
        r_pt = np.linalg.norm(th1 - mul(At, th1))
        r_dp = 0.7 * np.linalg.norm((p1 - p0) - mul(Ap, p1 - p0))
        r_dt = 3.0 * np.linalg.norm(mul(At, th1 - th0))
        want = [np.hypot(r_pp, r_pt), np.hypot(r_dp, r_dt), r_pp, r_pt, r_dp, r_dt]
        np.testing.assert_allclose(ora.res, want, rtol=1e-10, atol=1e-14)
        # v_bar = 0 at every node, every contingency and step (Section 3.2)
        np.testing.assert_allclose(node_mean(net, ora.v, phase=True), 0.0, atol=1e-11)


def test_tolerance_is_rms_scaled():
    ora = Oracle(make_case("tiny"), OracleOptions(eps=1e-4))
    n = ora.net
    assert n.J == 2 * n.L + n.S
    assert ora.tolerance() == pytest.approx(1e-4 * np.sqrt(2 * n.J * n.T * n.Kp))


def test_adaptation_rescales_scaled_duals():
    """At an adaptation the unscaled duals rho*u and rho*v are unchanged (Section 3.5)."""
    case = make_case(scale_case(14, 4, 2, seed=11))
    ora = Oracle(case, OracleOptions(adapt_every=10, rho_p=1.0, rho_theta=1.0))
    for _ in range(9):
        ora.step()
    # run the 10th step by hand without adaptation, then compare
    shadow = Oracle(case, OracleOptions(adapt_every=0, rho_p=1.0, rho_theta=1.0))
    for _ in range(10):
        shadow.step()
    ora.step()
    assert ora.rho_history and ora.rho_history[0][0] == 10
    np.testing.assert_allclose(ora.rho_p * ora.u, shadow.rho_p * shadow.u, atol=1e-12)
    np.testing.assert_allclose(ora.rho_th * ora.v, shadow.rho_th * shadow.v, atol=1e-12)
    assert (ora.rho_p, ora.rho_th) != (1.0, 1.0)


@pytest.mark.parametrize("part", ["p", "theta"])
def test_adaptive_rule_direction_per_part(part):
    """Section 3.5's case rule, pinned directly on residual pairs built on
    each side of mu: a primal part above mu times its dual part multiplies
    that part's penalty by gamma, a dual part above mu times the primal part
    divides it by gamma, anything in between (including equality at mu,
    the comparisons being strict) keeps it.  The other part's penalty is left
    alone, and the scaled duals of the changed part are multiplied by
    rho_old / rho_new (u for power, v for phase)."""
    mu, gamma = 2.0, 1.1
    case = make_case(scale_case(14, 4, 2, seed=11))
    cases = [((3.0, 1.0), gamma), ((2.0 + 1e-9, 1.0), gamma), ((2.0, 1.0), 1.0), ((1.5, 1.0), 1.0),
             ((1.0, 1.0), 1.0), ((1.0, 2.0), 1.0), ((1.0, 2.0 + 1e-9), 1 / gamma), ((1.0, 5.0), 1 / gamma),
             ((0.0, 0.0), 1.0)]
    for (rprim, rdual), factor in cases:
        ora = Oracle(case, OracleOptions(adapt_every=10, mu=mu, gamma=gamma, rho_p=0.7, rho_theta=3.0))
        for _ in range(3):
            ora.step()
        u0, v0 = ora.u.copy(), ora.v.copy()
        # the other part sits exactly at balance (both zero): never changes
        if part == "p":
            ora._adapt(rprim, 0.0, rdual, 0.0)
            assert ora.rho_p == pytest.approx(0.7 * factor, rel=1e-15), (rprim, rdual)
            assert ora.rho_th == 3.0
            np.testing.assert_allclose(ora.u, u0 / factor, rtol=1e-14, atol=0)
            np.testing.assert_array_equal(ora.v, v0)
        else:
            ora._adapt(0.0, rprim, 0.0, rdual)
            assert ora.rho_th == pytest.approx(3.0 * factor, rel=1e-15), (rprim, rdual)
            assert ora.rho_p == 0.7
            np.testing.assert_allclose(ora.v, v0 / factor, rtol=1e-14, atol=0)
            np.testing.assert_array_equal(ora.u, u0)
