"""Pins for the oracle's device proximal operators (CPU only).

Each prox is checked against something other than its own formula:
golden-section minimisation of the prox objective written from the device
cost of Section 2.1, an exhaustive active-set solve of the quadratic program
of Eq. (prox-general-form), and the closed form of a one-step battery.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import (inner_admm, inner_matrix, prox_fixed_load, prox_gen, prox_hvdc, prox_line,
                    ramp_rows, storage_rows)
from oracle.mp import storage_layout

GR = (math.sqrt(5.0) - 1.0) / 2.0


def golden(f, lo, hi, iters=200):
    """Minimise a 1-D convex function on [lo, hi] by golden-section search."""
    a, b = lo, hi
    c, d = b - GR * (b - a), a + GR * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(iters):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - GR * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + GR * (b - a)
            fd = f(d)
    return 0.5 * (a + b)


# --------------------------------------------------------------------------
# generator / curtailable load / fixed load (Section 2.1, Section 4.2)
# --------------------------------------------------------------------------

def test_prox_gen_matches_brute_force(rng):
    for _ in range(300):
        a = rng.uniform(0.0, 0.2)
        b = rng.uniform(-50, 50)
        pmin = rng.uniform(-2, 1)
        pmax = pmin + rng.uniform(0.0, 3)
        rho = rng.uniform(0.05, 60)
        x = rng.normal(0, 3)

        def obj(p):
            return a * p * p + b * p + 0.5 * rho * (p - x) ** 2

        ref = golden(obj, pmin, pmax)
        got = prox_gen(x, a, b, pmin, pmax, rho)
        assert abs(got - ref) <= 1e-6 * max(1.0, abs(ref))


def test_prox_curtailable_load_is_generator_on_negative_box(rng):
    # curtailable load: cost voll*(p + P) on [-P, 0] (Section 2.1: pmin < pmax <= 0)
    for _ in range(100):
        P, voll, rho, x = rng.uniform(0.1, 2), rng.uniform(1, 600), rng.uniform(0.1, 50), rng.normal(0, 2)
        ref = golden(lambda p: voll * (p + P) + 0.5 * rho * (p - x) ** 2, -P, 0.0)
        assert abs(prox_gen(x, 0.0, voll, -P, 0.0, rho) - ref) <= 1e-6


def test_prox_fixed_load():
    x = np.array([0.3, -7.0, 2.0])
    np.testing.assert_array_equal(prox_fixed_load(x, np.array([1.0, 0.5, 0.0])), [-1.0, -0.5, -0.0])


# --------------------------------------------------------------------------
# DC line (Section 2.1 f^ac), brute force over (p2, theta2)
# --------------------------------------------------------------------------

def _line_brute(x1, x2, y1, y2, u, b, rp, rt):
    # feasible set of f^ac parametrised by p2 in [-u, u] and theta2 (theta1 = theta2 + p2/b)
    def inner(p2):
        def g(t2):
            t1 = t2 + p2 / b
            return rt / 2 * ((t1 - y1) ** 2 + (t2 - y2) ** 2)
        span = 10 + abs(y1) + abs(y2) + abs(p2 / b)
        t2 = golden(g, -span, span)
        return t2, rp / 2 * ((-p2 - x1) ** 2 + (p2 - x2) ** 2) + g(t2)

    p2 = golden(lambda q: inner(q)[1], -u, u)
    t2 = inner(p2)[0]
    return -p2, p2, t2 + p2 / b, t2


@pytest.mark.parametrize("seed", range(40))
def test_prox_line_matches_brute_force(seed):
    r = np.random.default_rng(seed)
    x1, x2, y1, y2 = r.normal(0, 2, 4)
    u = r.uniform(0.05, 3)
    b = r.uniform(0.5, 25)
    rp, rt = r.uniform(0.1, 20), r.uniform(0.1, 200)
    ref = _line_brute(x1, x2, y1, y2, u, b, rp, rt)
    got = prox_line(x1, x2, y1, y2, u, b, rp, rt, True)
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-7)


def test_prox_line_flow_and_angle_relation(rng):
    x = rng.normal(0, 2, (4, 1000))
    u = rng.uniform(0.1, 2, 1000)
    b = rng.uniform(1, 20, 1000)
    p1, p2, t1, t2 = prox_line(*x, u, b, 2.0, 5.0, np.ones(1000, bool))
    np.testing.assert_allclose(p1 + p2, 0.0, atol=1e-15)
    assert np.all(np.abs(p2) <= u + 1e-15)
    np.testing.assert_allclose(p2, b * (t1 - t2), rtol=1e-12, atol=1e-14)


def test_prox_line_outage_decouples():
    # contingency parameters u = b = 0 (Section 2.3): no flow, angles follow their targets
    p1, p2, t1, t2 = prox_line(0.7, -0.2, 0.3, -0.4, 0.0, 0.0, 1.0, 1.0, False)
    assert (p1, p2, t1, t2) == (0.0, 0.0, 0.3, -0.4)


@pytest.mark.parametrize("seed", range(20))
def test_prox_hvdc_matches_brute_force(seed):
    # HVDC link (Section 2.1, other devices): p1 + p2 = 0, |p2| <= u, no angle
    r = np.random.default_rng(100 + seed)
    x1, x2 = r.normal(0, 2, 2)
    u = r.uniform(0.05, 3)
    rho = r.uniform(0.1, 50)
    p2 = golden(lambda q: rho / 2 * ((-q - x1) ** 2 + (q - x2) ** 2), -u, u)
    got = prox_hvdc(x1, x2, u)
    np.testing.assert_allclose(got, (-p2, p2), rtol=1e-6, atol=1e-7)


# --------------------------------------------------------------------------
# iterative proxes (Appendix D) vs the exact prox by exhaustive active sets
# --------------------------------------------------------------------------

def _qp_active_set(H, g, A, h, eq, tol=1e-9):
    """Exact minimiser of 0.5 z'Hz + g'z s.t. A z <= h (== on eq rows), H > 0,
    by enumerating inequality active sets and checking KKT."""
    ineq = np.nonzero(~eq)[0]
    eqr = np.nonzero(eq)[0]
    n = H.shape[0]
    # a row and its negation (two sides of one box) are never both active
    opposite = {(i, j) for i in ineq for j in ineq if i < j and np.allclose(A[i], -A[j])}
    best = None
    for k in range(len(ineq) + 1):
        for act in itertools.combinations(ineq, k):
            if any((i, j) in opposite for i, j in itertools.combinations(act, 2)):
                continue
            rows = np.concatenate([eqr, np.asarray(act, int)]).astype(int)
            Aw = A[rows]
            KKT = np.block([[H, Aw.T], [Aw, np.zeros((len(rows), len(rows)))]])
            rhs = np.concatenate([-g, h[rows]])
            try:
                sol = np.linalg.solve(KKT, rhs)
            except np.linalg.LinAlgError:
                continue
            if not np.all(np.isfinite(sol)):
                continue
            z, lam = sol[:n], sol[n:]
            if np.linalg.norm(KKT @ sol - rhs) > 1e-8 * (1 + np.linalg.norm(rhs)):
                continue
            if np.any(A[~eq] @ z > h[~eq] + tol) or np.any(np.abs(A[eq] @ z - h[eq]) > tol):
                continue
            if np.any(lam[len(eqr):] < -tol):
                continue
            best = z
            return best
    return best


def _ramp_exact(x, a, bc, pmin, pmax, R, rho):
    A, h, eq = ramp_rows(pmin, pmax, R)
    T = len(x)
    H = (2 * a + rho) * np.eye(T)
    g = bc * np.ones(T) - rho * x
    return _qp_active_set(H, g, A, h, eq)


@pytest.mark.parametrize("seed", range(12))
def test_ramp_inner_admm_converges_to_exact_prox(seed):
    r = np.random.default_rng(100 + seed)
    T = 3
    a, bc = r.uniform(0.01, 0.1), r.uniform(10, 40)
    pmax = np.full(T, r.uniform(1, 3))
    pmin = np.zeros(T)
    R = 0.2 * pmax[0]
    rho = r.uniform(5, 60)
    x = r.uniform(-0.5, 3.5, T)
    exact = _ramp_exact(x, a, bc, pmin, pmax, R, rho)
    A, h, eq = ramp_rows(pmin, pmax, R)
    Minv = np.linalg.inv(inner_matrix(np.full((1, T), a), rho, rho, A, T))
    z, _, _ = inner_admm(x[None], A, h[None], eq, np.full((1, T), bc), rho, rho, Minv,
                         np.zeros((1, len(h))), np.zeros((1, len(h))), 20000)
    np.testing.assert_allclose(z[0], exact, atol=1e-7)


def _storage_exact(x, eff, P, dur, cost, rho):
    T = len(x)
    A, h, eq = storage_rows(T, eff, P, dur)
    n = 4 * T + 1
    H = np.zeros((n, n))
    H[np.arange(T), np.arange(T)] = rho
    H += 1e-12 * np.eye(n)      # the prox makes p unique; (c, delta, s) follow from the equalities
    g = np.zeros(n)
    g[:T] = -rho * x
    g[storage_layout(T)[2]] = cost
    return _qp_active_set(H, g, A, h, eq, tol=1e-7)


@pytest.mark.parametrize("seed", range(6))
def test_storage_inner_admm_converges_to_exact_prox(seed):
    r = np.random.default_rng(200 + seed)
    T = 2
    eff, P, dur, cost = 0.95, r.uniform(0.5, 2), 4.0, r.uniform(0, 1)
    rho = r.uniform(5, 30)
    x = r.normal(0, 1.0, T)
    exact = _storage_exact(x, eff, P, dur, cost, rho)
    assert exact is not None
    A, h, eq = storage_rows(T, eff, P, dur)
    n = 4 * T + 1
    Minv = np.linalg.inv(inner_matrix(np.zeros((1, n)), rho, rho, A, T))
    q = np.zeros((1, n))
    q[0, storage_layout(T)[2]] = cost
    z, _, _ = inner_admm(x[None], A, h[None], eq, q, rho, rho, Minv,
                         np.zeros((1, len(h))), np.zeros((1, len(h))), 30000)
    np.testing.assert_allclose(z[0, :T], exact[:T], atol=1e-6)


@pytest.mark.parametrize("x", [0.0, 0.4, 3.0, -0.3, -2.0])
def test_storage_one_step_closed_form(x):
    # T = 1: s_1 = s_2 = 0 force delta = eff c, so p = (eff - 1) c <= 0, cost*eff*c;
    # the prox minimises cost eff c + rho/2 ((eff-1) c - x)^2 over 0 <= c <= P (eff c <= P too)
    eff, P, cost, rho = 0.9, 1.5, 0.3, 8.0
    c = np.clip(((eff - 1) * x * rho - cost * eff) / (rho * (eff - 1) ** 2), 0.0, P)
    want = (eff - 1) * c
    A, h, eq = storage_rows(1, eff, P, 4.0)
    Minv = np.linalg.inv(inner_matrix(np.zeros((1, 5)), rho, rho, A, 1))
    q = np.zeros((1, 5))
    q[0, 2] = cost
    z, _, _ = inner_admm(np.array([[x]]), A, h[None], eq, q, rho, rho, Minv,
                         np.zeros((1, len(h))), np.zeros((1, len(h))), 40000)
    assert abs(z[0, 0] - want) < 1e-6
    if x >= 0:
        assert abs(z[0, 0]) < 1e-6


def test_storage_rows_encode_the_battery():
    # a hand-built feasible schedule satisfies every row; perturbing the SoC breaks one
    T, eff, P, dur = 3, 0.9, 1.0, 2.0
    c = np.array([1.0, 0.0, 0.0])
    d = np.array([0.0, 0.5, 0.4])
    s = np.array([0.0, 0.9, 0.4, 0.0])
    p = d - c
    z = np.concatenate([p, c, d, s])
    A, h, eq = storage_rows(T, eff, P, dur)
    r = A @ z - h
    assert np.all(np.abs(r[eq]) < 1e-12) and np.all(r[~eq] <= 1e-12)
    z2 = z.copy()
    z2[3 * T + 2] += 0.1
    r2 = A @ z2 - h
    assert np.any(np.abs(r2[eq]) > 1e-3)


def test_inner_matrix_is_the_x_update_hessian(rng):
    # M must be the Hessian of z'Qz + rho/2||z_p - x||^2 + omega/2 ||A z - r||^2
    T = 4
    A, h, eq = ramp_rows(np.zeros(T), np.ones(T), 0.3)
    a, rho, omega = 0.07, 3.0, 5.0
    M = inner_matrix(np.full((1, T), a), rho, omega, A, T)[0]
    r = rng.normal(size=len(h))
    x = rng.normal(size=T)

    def F(z):
        return a * z @ z + rho / 2 * np.sum((z - x) ** 2) + omega / 2 * np.sum((A @ z - r) ** 2)

    e = 1e-4
    Hn = np.zeros((T, T))
    z0 = rng.normal(size=T)
    for i in range(T):
        for j in range(T):
            ei, ej = np.eye(T)[i] * e, np.eye(T)[j] * e
            Hn[i, j] = (F(z0 + ei + ej) - F(z0 + ei - ej) - F(z0 - ei + ej) + F(z0 - ei - ej)) / (4 * e * e)
    np.testing.assert_allclose(M, Hn, rtol=1e-5, atol=1e-5)
