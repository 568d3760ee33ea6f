"""Pins of the PyTorch unrolled reference (oracle/unrolled.py): it repeats the
NumPy oracle's iterates; its autograd gradients match central finite
differences; and with more iterations the gradient of the cost with respect
to a fixed load moves toward the nodal price (Section 5.5: the derivative of
the optimal cost with respect to the data is the dual variable)."""
import numpy as np
import pytest
import torch

from gridgen import make_case, scale_case
from oracle import Oracle, OracleOptions
from oracle.unrolled import Unrolled


def _case():
    return make_case(scale_case(40, 3, 2, seed=5, ramp=False, stor_per_node=0.0, fixed_frac=0.3))


def _case_inner():
    """Ramp-limited generators and batteries, whose prox is the inner ADMM,
    and two HVDC links."""
    return make_case(scale_case(40, 6, 2, seed=7, ramp=True, stor_per_node=0.1, fixed_frac=0.3, n_hvdc=2))


@pytest.mark.parametrize("inner", [False, True])
def test_repeats_the_oracle_iterates(inner):
    case = _case_inner() if inner else _case()
    ur = Unrolled(case, rho_p=1.0, rho_theta=2.0)
    f, pd = ur.run(ur.params(requires_grad=False), 17)
    o = Oracle(case, OracleOptions(adapt_every=0, eps=0.0, rho_theta=2.0))
    o.iterate(17, stop=False)
    np.testing.assert_allclose(pd.numpy(), o.dev_p(), rtol=1e-12, atol=1e-12)
    assert float(f) == pytest.approx(o.objective(), rel=1e-12)


@pytest.mark.parametrize("inner", [False, True])
def test_gradients_match_finite_differences(inner):
    """At these penalties 40 iterations reach a state where loads are served,
    some generators sit at capacity and some lines at their limit, so every
    gradient path is active (with ``inner``, through the inner ADMM of ramp
    generators and batteries); entries with a nonzero gradient are checked
    first, then a few zero ones."""
    case = _case_inner() if inner else _case()
    K = 40
    ur = Unrolled(case, rho_p=10.0, rho_theta=20.0)
    prm = ur.params()
    f, _ = ur.run(prm, K)
    f.backward()
    rng = np.random.default_rng(0)
    h = 1e-7
    checked = nonzero = 0
    for name, p in prm.items():
        g = p.grad.numpy().ravel()
        flat = p.detach().numpy().ravel()
        nz = np.flatnonzero(g)
        assert nz.size > 0, name
        zero = np.flatnonzero(g == 0)
        pick = list(rng.choice(nz, size=min(6, nz.size), replace=False))
        pick += list(rng.choice(zero, size=min(2, zero.size), replace=False)) if zero.size else []
        for j in pick:
            vals = []
            for s in (1, -1):
                q = {k: v.detach().clone() for k, v in prm.items()}
                q[name].view(-1)[j] += s * h
                vals.append(float(ur.run(q, K)[0]))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - g[j]) <= 1e-4 * (1 + abs(fd)), (name, j, fd, g[j])
            checked += 1
            nonzero += g[j] != 0
    assert checked >= 15 and nonzero >= 10


@pytest.mark.slow
def test_load_gradient_approaches_the_price_with_more_iterations():
    """Section 5.5: unrolling more iterations gives derivatives closer to the
    duality value; for a fixed load that value is the price at its node."""
    case = make_case("tiny")                 # fixed loads, T = 1
    ur = Unrolled(case, rho_p=1.0, rho_theta=10.0)
    errs = []
    for K in (2000, 6000):
        prm = ur.params()
        f, _ = ur.run(prm, K)
        f.backward()
        o = Oracle(case, OracleOptions(adapt_every=0, rho_theta=10.0, eps=0.0))
        o.iterate(K, stop=False)
        want = o.prices()[np.asarray(case["load_node"]), 0]
        errs.append(np.linalg.norm(prm["load_p"].grad.numpy()[:, 0] - want) / np.linalg.norm(want))
    assert errs[1] < 0.5 * errs[0]
