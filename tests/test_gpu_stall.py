"""The penalty limit, the stall rule and the residual history on the GPU,
against the oracle (neither the limit nor the rule is in the paper; the
options are documented in include/opf.h).

* the residual history rows equal the oracle's residuals and penalties at
  every iteration that forms them, and the ring keeps the latest rows;
* adapt_until: iterates and penalties equal the oracle's;
* a 40-bus instance on which the adaptive penalty cycles: the stall rule
  fixes the penalties, the run converges to the oracle's objective;
* an infeasible instance (fixed load above generation capacity) stops with
  OPF_ESTALLED, alone and inside a batch beside a feasible one; the next
  call continues.
"""
import numpy as np
import pytest

from gridgen import make_case, scale_case
from helpers import compare_residuals, compare_states, oracle_arrays
from oracle import Oracle, OracleOptions

pytestmark = pytest.mark.gpu

OPF_ESTALLED = 7
HF_CONVERGED, HF_ADAPTED, HF_FROZEN, HF_STALLED = 1, 2, 4, 8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2410_17203_gb300 import load_library
    load_library()


def _infeasible_tiny():
    case = make_case("tiny")
    cap = case["gen_pmax"].sum(axis=0)
    case["load_p"] = case["load_p"] * (1.5 * cap / case["load_p"].sum(axis=0))[None, :]
    return case


def test_history_rows_match_the_oracle_and_the_ring_keeps_the_latest():
    from paper_2410_17203_gb300 import Solver
    case = make_case(scale_case(150, 24, 6, seed=21))
    opts = dict(adapt_every=10, eps=1e-6, check_every=10)
    s = Solver(case, opts)
    s.iterate(120)
    hist = s.history()
    info = s.get_info()
    s.close()
    o = Oracle(case, OracleOptions(**opts))
    rows = []
    for _ in range(120):
        rho = (o.rho_p, o.rho_th)
        o.iterate(1, stop=False)
        if o.it % 10 == 0:
            scale = max(np.linalg.norm(a) for a in oracle_arrays(o).values())
            rows.append((o.it, o.res.copy(), rho, (o.rho_p, o.rho_th) != rho, scale))
    assert info["history_rows"] == len(rows) == len(hist) == 12
    for h, (it, res, rho, changed, scale) in zip(hist, rows):
        assert int(h[0]) == it
        compare_residuals(h[1:7], res, scale)
        assert (h[7], h[8]) == pytest.approx(rho, rel=1e-12)
        assert bool(int(h[9]) & HF_ADAPTED) == changed
    # a ring of 4 rows: the latest four, oldest first
    s = Solver(case, dict(opts, history_len=4))
    s.iterate(70)
    s.iterate(50)
    h4 = s.history()
    s.close()
    assert [int(r[0]) for r in h4] == [90, 100, 110, 120]
    np.testing.assert_array_equal(h4, hist[-4:])


def test_adapt_until_matches_the_oracle():
    from paper_2410_17203_gb300 import Solver
    case = make_case(scale_case(150, 24, 6, seed=21))
    opts = dict(adapt_every=10, eps=0.0, adapt_until=40)
    s = Solver(case, opts)
    s.iterate(100)
    st, info = s.state(), s.get_info()
    s.close()
    o = Oracle(case, OracleOptions(**opts))
    o.iterate(100, stop=False)
    assert len(o.rho_history) == 4
    compare_states(st, o)
    assert (info["rho_p"], info["rho_theta"]) == pytest.approx((o.rho_p, o.rho_th), rel=1e-12)


def test_cycling_instance_converges_with_the_stall_rule():
    from paper_2410_17203_gb300 import Solver
    case = make_case(scale_case(40, 12, 4, seed=22, stor_per_node=0.1))
    opts = dict(adapt_every=10, eps=1e-4, stall_window=300)
    s = Solver(case, opts)
    s.iterate(20000)
    info, sol, hist = s.get_info(), s.solution(), s.history()
    _, status = __import__("paper_2410_17203_gb300").opf_residuals(s.h, raise_on_status=False)
    s.close()
    o = Oracle(case, OracleOptions(**opts))
    o.iterate(20000)
    assert o.converged and o.frozen_at > 0
    assert status == 0 and info["converged"] == 1 and info["stalled"] == 0
    assert info["frozen_at"] > 0
    flags = hist[:, 9].astype(int)
    assert ((flags & HF_FROZEN) != 0).sum() == 1 and flags[-1] & HF_CONVERGED
    # no penalty change after the freeze
    frozen_row = int(np.nonzero(flags & HF_FROZEN)[0][0])
    assert not (flags[frozen_row:] & HF_ADAPTED).any()
    assert np.all(hist[frozen_row:, 7] == hist[frozen_row, 7])
    assert sol["objective"] == pytest.approx(o.objective(), rel=1e-4)


@pytest.mark.parametrize("adapt", [0, 10])
def test_infeasible_instance_reports_a_stall(adapt):
    from paper_2410_17203_gb300 import Solver, opf_residuals
    case = _infeasible_tiny()
    opts = dict(adapt_every=adapt, eps=1e-4, rho_theta=10.0, stall_window=400)
    s = Solver(case, opts)
    try:
        s.iterate(50000)
        res, status = opf_residuals(s.h, raise_on_status=False)
        info = s.get_info()
        assert status == OPF_ESTALLED and info["stalled"] == 1 and info["converged"] == 0
        assert info["iterations"] < 50000
        assert (info["frozen_at"] > 0) == (adapt > 0)
        assert int(s.history(1)[0, 9]) & HF_STALLED
        o = Oracle(case, OracleOptions(**opts))
        o.iterate(50000)
        assert o.stalled
        # the power-balance part of the primal residual: bounded below by the deficit
        deficit = case["load_p"].sum(axis=0) - case["gen_pmax"].sum(axis=0)
        lower = np.sqrt(o.net.Kp * np.sum(deficit ** 2) / o.net.J)
        assert res[2] >= 0.99 * lower
        # the next call restarts the window and iterates again
        it = info["iterations"]
        s.iterate(10)
        _, status = opf_residuals(s.h, raise_on_status=False)
        assert status == 0 and s.get_info()["iterations"] == it + 10
    finally:
        s.close()


def test_batch_counts_converged_and_stalled_instances():
    """Each instance keeps its own options: the infeasible one with the stall
    rule, the feasible one without (at fixed penalties it converges, slowly
    enough that a short window would call it stalled too)."""
    from paper_2410_17203_gb300 import (opf_batch_create, opf_batch_destroy, opf_batch_iterate,
                                        opf_batch_stopped, opf_create, opf_destroy, opf_get_info)
    opts = dict(adapt_every=0, eps=1e-4, rho_theta=10.0)
    hs = [opf_create(_infeasible_tiny(), dict(opts, stall_window=400)), opf_create(make_case("tiny"), opts)]
    b = opf_batch_create(hs)
    try:
        for _ in range(50):
            opf_batch_iterate(b, 1000)
            if sum(opf_batch_stopped(b)) == 2:
                break
        assert opf_batch_stopped(b) == (1, 1, 0)
        i0, i1 = opf_get_info(hs[0]), opf_get_info(hs[1])
        assert i0["stalled"] == 1 and i1["converged"] == 1
        # a stalled instance stays stopped inside the batch
        it = i0["iterations"]
        opf_batch_iterate(b, 100)
        assert opf_get_info(hs[0])["iterations"] == it
    finally:
        opf_batch_destroy(b)
        for h in hs:
            opf_destroy(h)


def test_history_edge_cases():
    """No ring (history_len = 0): nothing is kept; no stopping test and no
    adaptation: one row per call, at its last iteration; no stopping test
    (eps = 0): the stall rule has nothing to look at and never acts."""
    from paper_2410_17203_gb300 import Solver
    case = make_case("tiny")
    s = Solver(case, dict(eps=1e-4, history_len=0))
    try:
        s.iterate(30)
        assert s.get_info()["history_rows"] == 0 and len(s.history()) == 0
    finally:
        s.close()
    s = Solver(case, dict(eps=0.0, adapt_every=0, check_every=0, stall_window=10))
    try:
        for n in (7, 5, 9):
            s.iterate(n)
        h = s.history()
        assert [int(r[0]) for r in h] == [7, 12, 21]
        info = s.get_info()
        assert info["stalled"] == 0 and info["frozen_at"] == 0
    finally:
        s.close()
