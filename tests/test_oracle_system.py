"""System-level pins of the oracle at convergence (CPU only).

The converged message-passing iterate must be the optimum of the
contingency-constrained DC OPF, Eq. (contingency-dispatch), computed here by
means that share nothing with the method: bisection on the merit order for a
single bus, a hand-derived 3-bus optimum (Fig. 1 topology), and a generic
SLSQP solve of the DC OPF written in shift-factor form per contingency.
"""
import json
import os

import numpy as np
import pytest
from scipy.optimize import Bounds, LinearConstraint, minimize

from gridgen import make_case
from helpers import hang_triangle
from oracle import Oracle, OracleOptions

HERE = os.path.dirname(__file__)


def load_golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        d = json.load(f)
    case = {k: (np.asarray(v) if isinstance(v, list) else v) for k, v in d["case"].items()}
    case["outaged"] = np.asarray(case["outaged"], np.int32)
    return case, d["expected"]


def test_three_bus_congested_matches_analytic():
    case, exp = load_golden("three_bus_congested.json")
    o = Oracle(case, OracleOptions(adapt_every=0, rho_theta=100.0, eps=1e-9))
    o.iterate(100000)
    assert o.converged
    pd = o.dev_p()[:, 0]
    np.testing.assert_allclose(pd[:2], exp["gen_p"], atol=1e-6)
    np.testing.assert_allclose(pd[4:], exp["stor_p"], atol=1e-6)
    np.testing.assert_allclose(o.line_p()[0, :, 0], exp["line_flow"], atol=1e-6)
    np.testing.assert_allclose(o.prices()[:, 0], exp["price"], atol=1e-5)
    thb = o.thbar()[0, :, 0]
    assert thb[0] - thb[2] == pytest.approx(exp["angle_diff_n1_n3"], abs=1e-6)
    assert thb[0] - thb[1] == pytest.approx(exp["angle_diff_n1_n2"], abs=1e-6)
    assert thb[1] - thb[2] == pytest.approx(exp["angle_diff_n2_n3"], abs=1e-6)
    assert o.objective() == pytest.approx(exp["objective"], rel=1e-6)


def test_three_bus_golden_is_the_lp_optimum():
    """The hand-derived 3-bus values, re-derived by a linear program (HiGHS)
    over the generator outputs with shift-factor flow limits; the nodal
    prices are the LP cost's sensitivities to the load at each node."""
    from scipy.optimize import linprog
    case, exp = load_golden("three_bus_congested.json")
    N, fr, to, b, u = 3, case["line_from"], case["line_to"], case["line_b"], case["line_u"]
    inc = np.zeros((3, N))
    inc[np.arange(3), fr] = 1.0
    inc[np.arange(3), to] = -1.0
    Bbus = inc.T @ np.diag(b) @ inc
    X = np.zeros((N, N))
    X[1:, 1:] = np.linalg.inv(Bbus[1:, 1:])
    F = np.diag(b) @ inc @ X                            # flows = F @ injections
    C = np.zeros((N, 2))
    C[case["gen_node"], [0, 1]] = 1.0

    def solve(load):
        A = F @ C
        res = linprog(case["gen_b"], A_ub=np.vstack([A, -A]),
                      b_ub=np.concatenate([u + F @ load, u - F @ load]),
                      A_eq=np.ones((1, 2)), b_eq=[load.sum()], bounds=[(0, 5), (0, 5)], method="highs")
        assert res.status == 0
        return res.x, res.fun

    load = np.zeros(N)
    np.add.at(load, case["load_node"], case["load_p"][:, 0])
    g, f = solve(load)
    np.testing.assert_allclose(g, exp["gen_p"], atol=1e-9)
    assert f == pytest.approx(exp["objective"], abs=1e-9)
    flow = F @ (C @ g - load)
    np.testing.assert_allclose(flow, exp["line_flow"], atol=1e-9)
    assert flow[0] / b[0] == pytest.approx(exp["angle_diff_n1_n3"], abs=1e-12)
    assert flow[1] / b[1] == pytest.approx(exp["angle_diff_n1_n2"], abs=1e-12)
    assert flow[2] / b[2] == pytest.approx(exp["angle_diff_n2_n3"], abs=1e-12)
    h = 1e-4
    prices = [(solve(load + h * np.eye(N)[n])[1] - f) / h for n in range(N)]
    np.testing.assert_allclose(prices, exp["price"], atol=1e-6)


def _single_bus_case(rng, T=3):
    G, D = 5, 4
    pmax = rng.uniform(1, 3, G)
    return dict(
        n_nodes=1, T=T, line_from=np.zeros(0, np.int32), line_to=np.zeros(0, np.int32),
        line_b=np.zeros(0), line_u=np.zeros(0),
        gen_node=np.zeros(G, np.int32), gen_a=rng.uniform(0.01, 0.1, G), gen_b=rng.uniform(10, 40, G),
        gen_pmin=np.zeros((G, T)), gen_pmax=np.repeat(pmax[:, None], T, 1), gen_ramp=-np.ones(G),
        load_node=np.zeros(D, np.int32), load_p=rng.uniform(0.5, 1.5, (D, T)), load_voll=-np.ones(D),
        stor_node=np.zeros(0, np.int32), stor_P=np.zeros(0), stor_dur=np.zeros(0),
        stor_eff=np.zeros(0), stor_cost=np.zeros(0), outaged=np.zeros(0, np.int32))


def test_single_bus_economic_dispatch_matches_bisection(rng):
    case = _single_bus_case(rng)
    o = Oracle(case, OracleOptions(adapt_every=10, eps=1e-10))
    o.iterate(200000)
    assert o.converged
    a, b, pmax = case["gen_a"], case["gen_b"], case["gen_pmax"][:, 0]
    for t in range(case["T"]):
        demand = case["load_p"][:, t].sum()
        lo, hi = 0.0, 1000.0
        for _ in range(200):                       # merit-order bisection on the price
            lam = 0.5 * (lo + hi)
            if np.clip((lam - b) / (2 * a), 0, pmax).sum() > demand:
                hi = lam
            else:
                lo = lam
        want = np.clip((lam - b) / (2 * a), 0, pmax)
        np.testing.assert_allclose(o.dev_p()[:5, t], want, atol=1e-6)
        assert o.prices()[0, t] == pytest.approx(lam, abs=1e-5)


def _dcopf_slsqp(case):
    """Contingency-constrained DC OPF in shift-factor form, solved by SLSQP.

    Flows of contingency k are ``F_k (C g - d)`` with ``F_k`` the shift
    factors of the topology without the outaged line (reduced Laplacian
    inverse, node 0 as reference); variables are the generator outputs only.
    """
    N, T = case["n_nodes"], case["T"]
    assert T == 1 and len(case["stor_node"]) == 0
    G = len(case["gen_node"])
    # HVDC links: flow f_h from hvdc_from to hvdc_to, |f_h| <= u_h
    hf, ht = case.get("hvdc_from", np.zeros(0, int)), case.get("hvdc_to", np.zeros(0, int))
    H = len(hf)
    fr, to, bs, us = case["line_from"], case["line_to"], case["line_b"], case["line_u"]
    L = len(fr)
    out = case["outaged"]
    load = np.zeros(N)
    np.add.at(load, case["load_node"], case["load_p"][:, 0])
    C = np.zeros((N, G + H))                    # injections of the variables (g, f)
    C[case["gen_node"], np.arange(G)] = 1.0
    C[hf, G + np.arange(H)] -= 1.0
    C[ht, G + np.arange(H)] += 1.0
    Ain, bin_ = [], []
    for k in range(len(out) + 1):
        act = np.ones(L, bool)
        if k and out[k - 1] >= 0:
            act[out[k - 1]] = False
        inc = np.zeros((L, N))
        inc[np.arange(L), fr] = 1.0
        inc[np.arange(L), to] = -1.0
        inc = inc[act]
        Bl = np.diag(bs[act])
        Bbus = inc.T @ Bl @ inc
        Xr = np.zeros((N, N))
        Xr[1:, 1:] = np.linalg.inv(Bbus[1:, 1:])
        F = Bl @ inc @ Xr                       # flows = F @ injections
        Ain += [-(F @ C), F @ C]
        bin_ += [-us[act] - F @ load, -us[act] + F @ load]
    Ain = np.vstack(Ain)
    bin_ = np.concatenate(bin_)
    a = np.concatenate([case["gen_a"], np.zeros(H)])
    b = np.concatenate([case["gen_b"], np.zeros(H)])
    bal = np.concatenate([np.ones(G), np.zeros(H)])
    cons = [dict(type="eq", fun=lambda g: np.array([bal @ g - load.sum()]),
                 jac=lambda g: bal[None, :]),
            dict(type="ineq", fun=lambda g: Ain @ g - bin_, jac=lambda g: Ain)]
    bounds = [(case["gen_pmin"][g, 0], case["gen_pmax"][g, 0]) for g in range(G)]
    bounds += [(-case["hvdc_u"][h], case["hvdc_u"][h]) for h in range(H)]
    x0 = np.concatenate([np.full(G, load.sum() / G), np.zeros(H)])
    if H:
        # the zero-cost link flows make SLSQP's line search stall; an
        # interior-point solve handles them
        lb, ub = np.array([v[0] for v in bounds]), np.array([v[1] for v in bounds])
        res = minimize(lambda g: np.sum(a * g * g + b * g), x0, jac=lambda g: 2 * a * g + b,
                       hess=lambda g: np.diag(2 * a), method="trust-constr", bounds=Bounds(lb, ub),
                       constraints=[LinearConstraint(bal, load.sum(), load.sum()),
                                    LinearConstraint(Ain, bin_, np.inf)],
                       options=dict(gtol=1e-12, xtol=1e-14, maxiter=20000))
        assert res.status in (1, 2), res.message
        return res.x[:G], res.fun
    res = minimize(lambda g: np.sum(a * g * g + b * g), x0,
                   jac=lambda g: 2 * a * g + b, bounds=bounds, constraints=cons,
                   method="SLSQP", options=dict(maxiter=1000, ftol=1e-14))
    assert res.success, res.message
    return res.x[:G], res.fun


@pytest.fixture(scope="module")
def tiny_converged():
    case = make_case("tiny")
    o = Oracle(case, OracleOptions(adapt_every=0, rho_theta=10.0, eps=1e-8))
    o.iterate(200000)
    assert o.converged
    return case, o


def test_tiny_converges_to_independent_qp_optimum(tiny_converged):
    case, o = tiny_converged
    g, fopt = _dcopf_slsqp(case)
    assert o.objective() == pytest.approx(fopt, rel=1e-6)
    np.testing.assert_allclose(o.dev_p()[:len(g), 0], g, atol=2e-4)


def test_tiny_kkt_at_convergence(tiny_converged):
    case, o = tiny_converged
    net = o.net
    lam = o.prices()                          # [N, T]
    pg = o.dev_p()[:net.G]
    mc = 2 * net.gen_a[:, None] * pg + net.gen_b[:, None]
    price = lam[net.gen_node]
    inner = (pg > net.gen_pmin + 1e-6) & (pg < net.gen_pmax - 1e-6)
    np.testing.assert_allclose(mc[inner], price[inner], atol=1e-4)             # stationarity
    assert np.all(mc[pg >= net.gen_pmax - 1e-6] <= price[pg >= net.gen_pmax - 1e-6] + 1e-4)
    assert np.all(mc[pg <= net.gen_pmin + 1e-6] >= price[pg <= net.gen_pmin + 1e-6] - 1e-4)
    assert np.max(np.abs(o.pbar())) < 1e-7                                     # power balance
    pl = o.line_p()
    assert np.all(np.abs(pl) <= (net.line_u[None, :, None] * net.active[:, :, None]) + 1e-9)


def test_duplicate_no_outage_contingencies_keep_the_solution():
    base = make_case("tiny", K=0)
    dup = dict(base)
    dup["outaged"] = np.array([-1, -1, -1], np.int32)
    opts = OracleOptions(adapt_every=0, rho_theta=10.0, eps=1e-8)
    o0, o3 = Oracle(base, opts), Oracle(dup, opts)
    o0.iterate(200000)
    o3.iterate(200000)
    assert o0.converged and o3.converged
    np.testing.assert_allclose(o3.dev_p(), o0.dev_p(), atol=1e-5)
    assert o3.objective() == pytest.approx(o0.objective(), rel=2e-6)
    np.testing.assert_allclose(o3.prices(), o0.prices(), atol=1e-4)


def test_outage_of_a_zero_flow_line_keeps_the_solution():
    """Outaging a line that carries no power at the optimum changes no
    constraint that binds, so K such contingencies leave the dispatch, cost
    and prices of the base case (Eq. contingency-dispatch).  The line is the
    side X-Y of a triangle 0-X-Y hung on node 0 whose nodes X, Y have no
    devices: every flow in the triangle is zero, with or without the outage,
    and the outaged line is not a bridge."""
    base = make_case("tiny", K=0)
    n0 = base["n_nodes"]
    ext = hang_triangle(base)
    L = len(ext["line_b"])
    opts = OracleOptions(adapt_every=0, rho_theta=10.0, eps=1e-8)
    o0 = Oracle(base, opts)
    oe = Oracle(dict(ext, outaged=np.zeros(0, np.int32)), opts)
    ok = Oracle(dict(ext, outaged=np.array([L - 2] * 3, np.int32)), opts)
    for o in (o0, oe, ok):
        o.iterate(200000)
        assert o.converged
    for o in (oe, ok):
        np.testing.assert_allclose(o.dev_p(), o0.dev_p(), atol=1e-5)
        assert o.objective() == pytest.approx(o0.objective(), rel=2e-6)
        np.testing.assert_allclose(o.prices()[:n0], o0.prices(), atol=1e-4)
        np.testing.assert_allclose(o.line_p()[:, L - 3:], 0.0, atol=1e-6)
    # the outaged copies carry nothing on X-Y; the base row is the base case
    np.testing.assert_allclose(ok.line_p()[1:, L - 2], 0.0, atol=0)


def test_adaptive_penalty_keeps_the_fixed_point():
    base = make_case("tiny", K=0)
    fixed = Oracle(base, OracleOptions(adapt_every=0, rho_theta=10.0, eps=1e-8))
    adapt = Oracle(base, OracleOptions(adapt_every=10, eps=1e-8))
    fixed.iterate(200000)
    adapt.iterate(200000)
    assert fixed.converged and adapt.converged
    assert adapt.objective() == pytest.approx(fixed.objective(), rel=1e-7)
    np.testing.assert_allclose(adapt.dev_p(), fixed.dev_p(), atol=1e-5)


def _multiperiod_case(rng, T=6):
    G, D, B = 3, 3, 2
    pmax = rng.uniform(1.0, 2.0, G)
    t = np.arange(T)
    prof = 0.6 + 0.4 * np.sin(2 * np.pi * t / T)
    return dict(
        n_nodes=1, T=T, line_from=np.zeros(0, np.int32), line_to=np.zeros(0, np.int32),
        line_b=np.zeros(0), line_u=np.zeros(0),
        gen_node=np.zeros(G, np.int32), gen_a=rng.uniform(0.05, 0.3, G),
        gen_b=np.array([10.0, 20.0, 35.0]),
        gen_pmin=np.zeros((G, T)), gen_pmax=np.repeat(pmax[:, None], T, 1), gen_ramp=0.2 * pmax,
        load_node=np.zeros(D, np.int32), load_p=rng.uniform(0.9, 1.3, (D, 1)) * prof[None],
        load_voll=np.full(D, 500.0),
        stor_node=np.zeros(B, np.int32), stor_P=np.array([0.4, 0.3]), stor_dur=np.array([2.0, 3.0]),
        stor_eff=np.array([0.95, 0.9]), stor_cost=np.array([0.5, 1.0]),
        outaged=np.zeros(0, np.int32))


def _multiperiod_slsqp(case):
    """The same multi-period single-bus problem as one QP over
    (gen output, battery charge/discharge/state of charge, load served)."""
    T = case["T"]
    G, D, B = len(case["gen_node"]), len(case["load_node"]), len(case["stor_node"])
    ng, nc, nd, ns, nl = G * T, B * T, B * T, B * (T + 1), D * T
    o_g, o_c, o_d, o_s, o_l = 0, ng, ng + nc, ng + nc + nd, ng + nc + nd + ns
    nv = o_l + nl
    a, b, voll = case["gen_a"], case["gen_b"], case["load_voll"]
    P = case["load_p"]
    ig = lambda g, t: o_g + g * T + t
    ic = lambda k, t: o_c + k * T + t
    idl = lambda k, t: o_d + k * T + t
    is_ = lambda k, t: o_s + k * (T + 1) + t
    il = lambda d, t: o_l + d * T + t

    def f(x):
        g = x[o_g:o_c].reshape(G, T)
        dl = x[o_d:o_s].reshape(B, T)
        served = x[o_l:].reshape(D, T)
        return (np.sum(a[:, None] * g * g + b[:, None] * g) + np.sum(voll[:, None] * (P - served))
                + np.sum(case["stor_cost"][:, None] * dl))

    def grad(x):
        gr = np.zeros(nv)
        g = x[o_g:o_c].reshape(G, T)
        gr[o_g:o_c] = (2 * a[:, None] * g + b[:, None]).ravel()
        gr[o_d:o_s] = np.repeat(case["stor_cost"], T)
        gr[o_l:] = -np.repeat(voll, T)
        return gr

    Aeq, beq, Ain, bin_ = [], [], [], []
    for t in range(T):                          # power balance
        r = np.zeros(nv)
        for g in range(G):
            r[ig(g, t)] = 1
        for k in range(B):
            r[idl(k, t)], r[ic(k, t)] = 1, -1
        for d in range(D):
            r[il(d, t)] = -1
        Aeq.append(r)
        beq.append(0.0)
    for k in range(B):                          # state of charge
        eff = case["stor_eff"][k]
        for t in range(T):
            r = np.zeros(nv)
            r[is_(k, t + 1)], r[is_(k, t)], r[ic(k, t)], r[idl(k, t)] = 1, -1, -eff, 1
            Aeq.append(r)
            beq.append(0.0)
        for t in (0, T):
            r = np.zeros(nv)
            r[is_(k, t)] = 1
            Aeq.append(r)
            beq.append(0.0)
    for g in range(G):                          # ramps
        R = case["gen_ramp"][g]
        for t in range(T - 1):
            r = np.zeros(nv)
            r[ig(g, t + 1)], r[ig(g, t)] = 1, -1
            Ain += [-r, r]
            bin_ += [-R, -R]
    Aeq, beq, Ain, bin_ = map(np.asarray, (Aeq, beq, Ain, bin_))
    bounds = ([(0, case["gen_pmax"][g, t]) for g in range(G) for t in range(T)]
              + [(0, case["stor_P"][k]) for k in range(B) for t in range(T)] * 2
              + [(0, case["stor_dur"][k] * case["stor_P"][k]) for k in range(B) for t in range(T + 1)]
              + [(0, P[d, t]) for d in range(D) for t in range(T)])
    cons = [dict(type="eq", fun=lambda x: Aeq @ x - beq, jac=lambda x: Aeq),
            dict(type="ineq", fun=lambda x: Ain @ x - bin_, jac=lambda x: Ain)]
    x0 = np.zeros(nv)
    x0[o_l:] = P.ravel()                        # serve all load from a flat dispatch
    x0[o_g:o_c] = np.repeat(P.sum(0)[None] / G, G, 0).ravel()
    from scipy.optimize import Bounds, LinearConstraint
    lo = np.array([bd[0] for bd in bounds], float)
    hi = np.array([bd[1] for bd in bounds], float)
    H = np.zeros((nv, nv))
    H[np.arange(o_g, o_c), np.arange(o_g, o_c)] = 2 * np.repeat(a, T)
    res = minimize(f, x0, jac=grad, hess=lambda x: H, method="trust-constr",
                   bounds=Bounds(lo, hi),
                   constraints=[LinearConstraint(Aeq, beq, beq),
                                LinearConstraint(Ain, bin_, np.inf)],
                   options=dict(maxiter=20000, gtol=1e-12, xtol=1e-14))
    assert res.status in (1, 2), res.message
    return res.x[o_g:o_c].reshape(G, T), f(res.x)


def test_ramp_and_storage_iteration_converges_to_qp_optimum(rng):
    case = _multiperiod_case(np.random.default_rng(77))
    g_ref, f_ref = _multiperiod_slsqp(case)
    o = Oracle(case, OracleOptions(adapt_every=10, eps=1e-9))
    o.iterate(300000)
    assert o.converged
    assert o.rho_history                    # adaptation ran (rescaling the inner duals)
    assert o.objective() == pytest.approx(f_ref, rel=1e-5)
    np.testing.assert_allclose(o.dev_p()[:3], g_ref, atol=2e-4)


def test_two_areas_joined_by_hvdc_match_merit_order():
    """Two single-bus areas joined only by an HVDC link (Section 2.1, other
    devices): the cheap area exports up to the link limit, and each area's
    price is its own marginal generator's cost."""
    u = 0.7
    case = dict(
        n_nodes=2, T=1, line_from=np.zeros(0, np.int32), line_to=np.zeros(0, np.int32),
        line_b=np.zeros(0), line_u=np.zeros(0),
        gen_node=np.array([0, 1], np.int32), gen_a=np.array([0.5, 1.0]), gen_b=np.array([10.0, 30.0]),
        gen_pmin=np.zeros((2, 1)), gen_pmax=np.full((2, 1), 5.0), gen_ramp=-np.ones(2),
        load_node=np.array([0, 1], np.int32), load_p=np.array([[0.5], [2.0]]), load_voll=-np.ones(2),
        stor_node=np.zeros(0, np.int32), stor_P=np.zeros(0), stor_dur=np.zeros(0),
        stor_eff=np.zeros(0), stor_cost=np.zeros(0), outaged=np.zeros(0, np.int32),
        hvdc_from=np.array([0], np.int32), hvdc_to=np.array([1], np.int32), hvdc_u=np.array([u]))
    o = Oracle(case, OracleOptions(adapt_every=10, eps=1e-10))
    o.iterate(200000)
    assert o.converged
    # area 0 serves its load and the export u: g0 = 0.5 + 0.7 = 1.2 at price
    # 2 * 0.5 * 1.2 + 10 = 11.2; area 1 serves 2.0 - 0.7 = 1.3 at 2 * 1.0 * 1.3 + 30 = 32.6
    pd = o.dev_p()[:, 0]
    np.testing.assert_allclose(pd[:2], [1.2, 1.3], atol=1e-6)
    np.testing.assert_allclose(pd[4:], [-u, u], atol=1e-6)
    np.testing.assert_allclose(o.prices()[:, 0], [11.2, 32.6], atol=1e-4)


def test_tiny_with_hvdc_converges_to_independent_qp_optimum():
    case = make_case("tiny", n_hvdc=3)
    o = Oracle(case, OracleOptions(adapt_every=0, rho_theta=10.0, eps=1e-8))
    o.iterate(200000)
    assert o.converged
    g, fopt = _dcopf_slsqp(case)
    assert o.objective() == pytest.approx(fopt, rel=1e-6)
    np.testing.assert_allclose(o.dev_p()[:len(g), 0], g, atol=2e-4)


def test_over_relaxed_iteration_reaches_the_same_optimum(tiny_converged):
    """Section 3.6: alpha = 1.5 changes the path, not the fixed point."""
    case, o1 = tiny_converged
    o = Oracle(case, OracleOptions(adapt_every=0, rho_theta=10.0, eps=1e-8, alpha=1.5))
    o.iterate(200000)
    assert o.converged
    g, fopt = _dcopf_slsqp(case)
    assert o.objective() == pytest.approx(fopt, rel=1e-6)
    np.testing.assert_allclose(o.dev_p()[:len(g), 0], g, atol=2e-4)
    np.testing.assert_allclose(o.prices(), o1.prices(), rtol=1e-3)
