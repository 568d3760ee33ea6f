"""GPU path vs the FP64 oracle, element by element (normwise per state array).

All calls go through the C ABI (ctypes binding).  Sizes span several CTAs and
ragged tails; the cases cover the 128-bit path (T % 4 == 0) and the scalar
path, outages, K = 0, T = 1, fixed and curtailable loads, ramp-limited
generators and batteries (Appendix D inner ADMM), with and without the
adaptive penalty.
"""
import numpy as np
import pytest

from gridgen import make_case, scale_case
from helpers import compare_residuals, compare_states, hang_triangle, oracle_arrays, rel_err
from oracle import Oracle, OracleOptions

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2410_17203_gb300 import load_library
    load_library()


def run_both(case, n, **opts):
    from paper_2410_17203_gb300 import Solver
    s = Solver(case, dict(opts))
    s.iterate(n)
    st = s.state()
    res = s.residuals()
    info = s.get_info()
    s.close()
    o = Oracle(case, OracleOptions(**opts))
    o.iterate(n, stop=opts.get("eps", 1e-4) > 0)
    return st, res, info, o


def _line_only_nodes():
    base = make_case(scale_case(80, 12, 2, seed=27))
    ext = hang_triangle(base, node=5)
    xy = len(ext["line_b"]) - 2
    return dict(ext, outaged=np.array([xy, base["outaged"][0], xy, base["outaged"][1]], np.int32))


CASES = {
    "tiny": lambda: make_case("tiny"),
    "mixed_T24": lambda: make_case(scale_case(150, 24, 6, seed=21)),
    "scalar_T7": lambda: make_case(scale_case(90, 7, 3, seed=22, fixed_frac=0.3)),
    "K0_fixed": lambda: make_case(scale_case(70, 8, 0, seed=23, fixed_frac=0.5, stor_per_node=0.0)),
    "T1_outages": lambda: make_case(scale_case(120, 1, 9, seed=24, fixed_frac=0.2)),
    "dup_noout": lambda: dict(make_case(scale_case(60, 12, 0, seed=25)),
                              outaged=np.array([-1, -1], np.int32)),
    "hvdc_T24": lambda: make_case(scale_case(160, 24, 5, seed=26, n_hvdc=4)),
    "hvdc_tiny": lambda: make_case("tiny", n_hvdc=3),
    # nodes with line terminals only; one of them keeps a single active line
    "line_only_nodes": lambda: _line_only_nodes(),
    # horizons above 128 steps: the inner-ADMM state stays in global memory
    "long_T200": lambda: make_case(scale_case(40, 200, 2, seed=29)),
    "long_T150": lambda: make_case(scale_case(30, 150, 1, seed=30, stor_per_node=0.1, fixed_frac=0.3)),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("n", [1, 10, 100])
def test_iterates_match_oracle_no_adaptation(name, n):
    case = CASES[name]()
    st, res, info, o = run_both(case, n, adapt_every=0, eps=0.0, rho_theta=5.0)
    compare_states(st, o)
    scale = max(np.linalg.norm(a) for a in oracle_arrays(o).values())
    compare_residuals(res, o.res, scale)
    assert info["iterations"] == n


@pytest.mark.parametrize("name", ["tiny", "mixed_T24", "scalar_T7", "hvdc_T24"])
def test_iterates_and_penalties_match_with_adaptation(name):
    case = CASES[name]()
    n = 100
    st, res, info, o = run_both(case, n, adapt_every=10, eps=0.0)
    # the sequence of penalty decisions must agree
    assert info["rho_p"] == pytest.approx(o.rho_p, rel=1e-12)
    assert info["rho_theta"] == pytest.approx(o.rho_th, rel=1e-12)
    compare_states(st, o)


def test_split_launches_equal_one_launch():
    """Iterations split over several launches (deferred v, pending rescale,
    dual residual history carried on the device) give the same iterate."""
    from paper_2410_17203_gb300 import Solver
    case = CASES["mixed_T24"]()
    a = Solver(case, dict(adapt_every=10, eps=0.0))
    a.iterate(60)
    b = Solver(case, dict(adapt_every=10, eps=0.0))
    for n in (7, 3, 10, 1, 29, 10):
        b.iterate(n)
    sa, sb = a.state(), b.state()
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)
    np.testing.assert_array_equal(a.residuals(), b.residuals())


def test_state_import_then_step_matches_oracle():
    """Warm start (Section 3.4): an oracle state imported through the C ABI
    continues exactly like the oracle does from that state."""
    from paper_2410_17203_gb300 import Solver
    case = CASES["mixed_T24"]()
    o = Oracle(case, OracleOptions(adapt_every=0, eps=0.0, rho_theta=5.0))
    o.iterate(40, stop=False)
    ref = oracle_arrays(o)
    st = {k: v.astype(np.float32) for k, v in ref.items()}
    inner = []
    for r in range(len(o.ramp_idx)):
        inner += [o.ramp_lam[r], o.ramp_beta[r]]
    for b in range(o.net.B):
        inner += [o.stor_lam[b], o.stor_beta[b]]
    st["inner"] = np.concatenate(inner).astype(np.float32)
    s = Solver(case, dict(adapt_every=0, eps=0.0, rho_theta=5.0))
    s.set_state(st)
    back = s.state()
    for k in ref:
        assert rel_err(back[k], ref[k]) < 1e-6, k
    assert rel_err(back["inner"], st["inner"]) < 1e-6
    # continue both from the (FP32-rounded) state
    o2 = Oracle(case, OracleOptions(adapt_every=0, eps=0.0, rho_theta=5.0))
    o2.load_state(st)
    s.iterate(5)
    o2.iterate(5, stop=False)
    compare_states(s.state(), o2)


def test_solution_outputs_match_oracle():
    from paper_2410_17203_gb300 import Solver
    case = CASES["mixed_T24"]()
    s = Solver(case, dict(adapt_every=10, eps=0.0))
    s.iterate(80)
    sol = s.solution()
    o = Oracle(case, OracleOptions(adapt_every=10, eps=0.0))
    o.iterate(80, stop=False)
    assert rel_err(sol["p_dev"], o.dev_p()) < 1e-5
    assert rel_err(sol["p_line"], o.line_p()) < 1e-5
    assert rel_err(sol["theta_node"], o.thbar()) < 1e-5
    assert rel_err(sol["price"], o.prices()) < 1e-5
    assert sol["objective"] == pytest.approx(o.objective(), rel=1e-5)


def test_phase_dual_stays_zero_mean_per_node():
    """v_bar = 0 at every node and contingency (Section 3.2 invariant)."""
    from paper_2410_17203_gb300 import Solver
    case = CASES["mixed_T24"]()
    s = Solver(case, dict(adapt_every=10, eps=0.0))
    s.iterate(37)
    st = s.state()
    N = case["n_nodes"]
    Kp, L, T = st["v1"].shape
    acc = np.zeros((Kp, N, T))
    cnt = np.zeros(N)
    np.add.at(acc, (slice(None), case["line_from"]), st["v1"].astype(np.float64))
    np.add.at(acc, (slice(None), case["line_to"]), st["v2"].astype(np.float64))
    scale = np.abs(st["v1"]).max() + np.abs(st["v2"]).max()
    assert np.abs(acc).max() <= 1e-5 * scale * 8


def test_converged_objective_matches_oracle():
    """Both sides run to the Eq. (converge) tolerance; objectives within 1e-4."""
    from paper_2410_17203_gb300 import Solver
    case = make_case("tiny")
    opts = dict(adapt_every=0, rho_theta=10.0, eps=1e-4)
    s = Solver(case, opts)
    s.iterate(50000)
    info = s.get_info()
    res = s.residuals()
    assert info["converged"] == 1
    assert max(res[0], res[1]) <= info["tolerance"]
    sol = s.solution()
    o = Oracle(case, OracleOptions(**opts))
    o.iterate(50000)
    assert o.converged
    assert sol["objective"] == pytest.approx(o.objective(), rel=1e-4)


@pytest.mark.parametrize("spec", [dict(n_nodes=30, T=24, K=4, seed=24, stor_per_node=0.1),
                                  dict(n_nodes=40, T=6, K=4, seed=21, stor_per_node=0.1)])
def test_converged_objective_matches_oracle_multiperiod(spec):
    """The setting the benchmark solves in: T > 1 with ramp-limited
    generators and batteries (Appendix D inner ADMM, whose discharge
    variable carries the storage cost), curtailable loads, four outages, the
    adaptive penalty every 10 iterations.  Both sides run to eps = 1e-4
    (Eq. converge); the objectives agree to 1e-4 relative and the GPU's
    primal residual is within the tolerance, i.e. at most 1e-4 per terminal
    in the RMS sense of Eq. (converge)."""
    from paper_2410_17203_gb300 import Solver
    case = make_case(scale_case(**spec))
    assert len(case["stor_node"]) > 0 and (case["gen_ramp"] >= 0).all() and case["T"] > 1
    opts = dict(adapt_every=10, eps=1e-4)
    s = Solver(case, opts)
    try:
        s.iterate(30000)
        info, res, sol = s.get_info(), s.residuals(), s.solution()
    finally:
        s.close()
    o = Oracle(case, OracleOptions(**opts))
    o.iterate(30000)
    assert o.converged and info["converged"] == 1
    assert max(res[0], res[1]) <= info["tolerance"]
    assert info["tolerance"] == pytest.approx(o.tolerance(), rel=1e-12)
    # primal residual per terminal (RMS over the 2 J T (K+1) entries) <= 1e-4
    d = info
    assert res[0] / np.sqrt(2.0 * d["J"] * d["T"] * (d["K"] + 1)) <= 1e-4
    assert sol["objective"] == pytest.approx(o.objective(), rel=1e-4)
    # the two sides stop within a few tests of each other
    assert abs(info["iterations"] - o.it) <= 0.1 * o.it


# ---------------------------------------------------------------------------
# failure detection without a GPU fault
# ---------------------------------------------------------------------------

def test_sync_timeout_is_reported_and_recoverable():
    """A synchronizing call that outlives sync_timeout_ms returns OPF_ETIMEOUT
    while the queued iterations keep running; a later call sees them done."""
    import time
    from paper_2410_17203_gb300 import Solver, opf_iterate, opf_residuals
    case = CASES["mixed_T24"]()
    s = Solver(case, dict(sync_timeout_ms=1, eps=0.0))
    n = 20000
    opf_iterate(s.h, n)
    _, st = opf_residuals(s.h, raise_on_status=False)
    assert st == 4                                   # OPF_ETIMEOUT, work still queued
    deadline = time.time() + 120
    while st == 4 and time.time() < deadline:
        time.sleep(0.05)
        _, st = opf_residuals(s.h, raise_on_status=False)
    assert st == 0
    assert s.get_info()["iterations"] == n
    s.close()


def test_nonfinite_state_is_reported():
    from paper_2410_17203_gb300 import Solver, opf_residuals
    case = CASES["mixed_T24"]()
    s = Solver(case, dict(eps=0.0))
    st = s.state()
    st["u"][0, 3, 2] = np.nan
    s.set_state(st)
    s.iterate(5)
    _, status = opf_residuals(s.h, raise_on_status=False)
    assert status == 5                               # OPF_ENONFINITE
    # found at the first iteration that forms residuals: here the call's last
    assert s.get_info()["iterations"] == 5
    s.iterate(5)                                     # a stopped context stays stopped
    assert s.get_info()["iterations"] == 5


def test_longest_horizon_matches_oracle():
    """T = 2048, the largest horizon the library takes: ramp-limited
    generators' inner ADMM over 2048 steps (work arrays of 192 KB of shared
    memory per CTA, state in global memory), with an outage."""
    case = make_case(scale_case(12, 2048, 1, seed=31, stor_per_node=0.0))
    st, res, info, o = run_both(case, 20, adapt_every=10, eps=0.0)
    compare_states(st, o)
    assert info["iterations"] == 20


def test_empty_and_degenerate_shapes():
    """One bus and no lines (no phase terminals), K = 0, T = 1."""
    from paper_2410_17203_gb300 import Solver
    rng = np.random.default_rng(3)
    G, D, T = 3, 2, 1
    case = dict(n_nodes=1, T=T, line_from=np.zeros(0, np.int32), line_to=np.zeros(0, np.int32),
                line_b=np.zeros(0), line_u=np.zeros(0), gen_node=np.zeros(G, np.int32),
                gen_a=rng.uniform(0.01, 0.1, G), gen_b=rng.uniform(10, 40, G),
                gen_pmin=np.zeros((G, T)), gen_pmax=np.full((G, T), 2.0), gen_ramp=-np.ones(G),
                load_node=np.zeros(D, np.int32), load_p=np.full((D, T), 0.8),
                load_voll=-np.ones(D), stor_node=np.zeros(0, np.int32), stor_P=np.zeros(0),
                stor_dur=np.zeros(0), stor_eff=np.zeros(0), stor_cost=np.zeros(0),
                outaged=np.zeros(0, np.int32))
    st, res, info, o = run_both(case, 30, adapt_every=10, eps=0.0)
    compare_states(st, o, keys=["p_dev", "u"])


# --------------------------------------------------------------------------
# over-relaxation (Section 3.6)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["tiny", "mixed_T24", "scalar_T7", "T1_outages", "hvdc_T24"])
@pytest.mark.parametrize("n", [1, 10, 100])
def test_over_relaxed_iterates_match_oracle(name, n):
    """alpha = 1.5: the device keeps relaxed schedules and rebuilds the
    actual iterate on export; the oracle runs the explicit-copy ADMM."""
    case = CASES[name]()
    st, res, info, o = run_both(case, n, adapt_every=0, eps=0.0, rho_theta=5.0, alpha=1.5)
    compare_states(st, o)
    scale = max(np.linalg.norm(a) for a in oracle_arrays(o).values())
    compare_residuals(res, o.res, scale)


@pytest.mark.parametrize("name", ["tiny", "mixed_T24"])
def test_over_relaxed_penalties_match_with_adaptation(name):
    case = CASES[name]()
    st, res, info, o = run_both(case, 100, adapt_every=10, eps=0.0, alpha=1.5)
    assert info["rho_p"] == pytest.approx(o.rho_p, rel=1e-12)
    assert info["rho_theta"] == pytest.approx(o.rho_th, rel=1e-12)
    compare_states(st, o)


def test_over_relaxed_split_launches_and_solution():
    """Relaxed state carried across launches; opf_solution's schedules and
    objective are those of the actual iterate."""
    from paper_2410_17203_gb300 import Solver
    case = CASES["mixed_T24"]()
    opts = dict(adapt_every=10, eps=0.0, alpha=1.5)
    a, b = Solver(case, opts), Solver(case, opts)
    try:
        a.iterate(37)
        for n in (5, 16, 1, 15):
            b.iterate(n)
        sa, sb = a.state(), b.state()
        for k in sa:
            np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)
        o = Oracle(case, OracleOptions(**opts))
        o.iterate(37, stop=False)
        sol = a.solution()
        assert sol["objective"] == pytest.approx(o.objective(), rel=1e-5)
        assert rel_err(sol["p_dev"], o.dev_p()) <= 1e-5
    finally:
        a.close()
        b.close()


def test_over_relaxed_converges_to_the_plain_optimum():
    from paper_2410_17203_gb300 import Solver
    case = CASES["tiny"]()
    base = dict(adapt_every=0, rho_theta=10.0, eps=1e-4)
    obj = []
    for alpha in (1.0, 1.5):
        s = Solver(case, dict(base, alpha=alpha))
        try:
            for _ in range(400):
                s.iterate(100)
                if s.get_info()["converged"]:
                    break
            assert s.get_info()["converged"]
            obj.append(s.solution()["objective"])
        finally:
            s.close()
    assert obj[1] == pytest.approx(obj[0], rel=1e-3)


def test_alpha_out_of_range_is_rejected():
    from paper_2410_17203_gb300 import OpfError, Solver
    for alpha in (0.9, 2.0):
        with pytest.raises(OpfError):
            Solver(CASES["tiny"](), dict(alpha=alpha))


def test_over_relaxed_state_import_restarts_the_copies():
    """With alpha != 1 an imported state restarts the duplicate variables at
    z = p~, xi = theta_bar on both sides (the device's relaxed schedules
    become the imported ones); the continuation then matches the oracle."""
    from paper_2410_17203_gb300 import Solver
    case = CASES["mixed_T24"]()
    opts = dict(adapt_every=0, eps=0.0, rho_theta=5.0, alpha=1.5)
    a = Solver(case, opts)
    b = Solver(case, opts)
    try:
        a.iterate(20)
        st = a.state()
        b.set_state(st)
        b.iterate(10)
        o = Oracle(case, OracleOptions(**opts))
        o.load_state({k: v.astype(np.float64) for k, v in st.items()})
        o.iterate(10, stop=False)
        compare_states(b.state(), o)
    finally:
        a.close()
        b.close()
