"""The penalty limit and the stall rule of the oracle (CPU only).

Neither is in the paper: Section 3.5 adapts the penalties for the whole run.
The residual balancing rule it takes from Boyd et al. (2011, Section 3.4.1)
keeps ADMM's convergence guarantee only when the penalty stops changing after
finitely many iterations, and on some instances the rule applied forever
cycles: the residuals come close to the tolerance, then grow again.

* ``adapt_until``: the run equals the unlimited one up to that iteration,
  and the penalties stay fixed afterwards;
* the stall rule fixes the penalties of a cycling run, which then converges
  to the optimum that fixed penalties reach from the start;
* an infeasible instance (fixed load above the generation capacity) stalls:
  with fixed penalties at once, with adaptive ones after fixing them first.
"""
import numpy as np
import pytest

from gridgen import make_case, scale_case
from oracle import Oracle, OracleOptions


def test_adapt_until_stops_the_penalty_changes():
    case = make_case(scale_case(30, 6, 3, seed=12))
    a = Oracle(case, OracleOptions(adapt_every=10, eps=0.0))
    b = Oracle(case, OracleOptions(adapt_every=10, eps=0.0, adapt_until=40))
    a.iterate(40, stop=False)
    b.iterate(40, stop=False)
    np.testing.assert_array_equal(a.p, b.p)
    np.testing.assert_array_equal(a.u, b.u)
    assert a.rho_history == b.rho_history and len(b.rho_history) == 4
    rho = (b.rho_p, b.rho_th)
    b.iterate(200, stop=False)
    assert (b.rho_p, b.rho_th) == rho and len(b.rho_history) == 4


def test_cycling_run_is_fixed_by_the_stall_rule_and_converges():
    """A 40-bus, T = 12 instance on which the adaptive penalty, applied every
    10 iterations for ever, never reaches eps = 1e-4 (residuals grow again
    after approaching it); with the stall rule the penalties are fixed at the
    first stall and the run converges to the fixed-penalty optimum."""
    case = make_case(scale_case(40, 12, 4, seed=22, stor_per_node=0.1))
    base = dict(adapt_every=10, eps=1e-4)
    cyc = Oracle(case, OracleOptions(**base))
    cyc.iterate(4000)
    assert not cyc.converged
    assert cyc.res.max() > 5 * cyc.tolerance()
    st = Oracle(case, OracleOptions(**base, stall_window=300))
    st.iterate(20000)
    assert st.converged and not st.stalled
    assert 0 < st.frozen_at < st.it
    assert all(h[0] < st.frozen_at for h in st.rho_history)
    fixed = Oracle(case, OracleOptions(adapt_every=0, eps=1e-4))
    fixed.iterate(20000)
    assert fixed.converged
    assert st.objective() == pytest.approx(fixed.objective(), rel=1e-3)


def _infeasible_tiny():
    case = make_case("tiny")
    cap = case["gen_pmax"].sum(axis=0)
    case["load_p"] = case["load_p"] * (1.5 * cap / case["load_p"].sum(axis=0))[None, :]
    assert (case["load_voll"] < 0).all()          # fixed loads: nothing can be shed
    return case


@pytest.mark.parametrize("adapt", [0, 10])
def test_infeasible_instance_stalls(adapt):
    case = _infeasible_tiny()
    o = Oracle(case, OracleOptions(adapt_every=adapt, eps=1e-4, rho_theta=10.0, stall_window=400))
    n = o.iterate(50000)
    assert o.stalled and not o.converged and n < 50000
    assert (o.frozen_at > 0) == (adapt > 0)
    # the power-balance part of the primal residual stays bounded away from 0:
    # at least the total deficit spread over the node terminals (each node's
    # mean |pbar_n| weighted by its |n| terminals; Cauchy-Schwarz)
    net = o.net
    deficit = case["load_p"].sum(axis=0) - case["gen_pmax"].sum(axis=0)
    lower = np.sqrt(net.Kp * np.sum(deficit ** 2) / net.J)
    assert o.res[2] >= 0.99 * lower
    # the next call restarts the window and runs again
    it = o.it
    o.iterate(10)
    assert o.it == it + 10 and not o.stalled
