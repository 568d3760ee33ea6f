"""Contingency slices (include/opf.h, opf_create_slice): the iteration split
over contexts that each hold a block of the contingencies and exchange one
buffer per iteration (Section 3.2's sums over k for the shared devices and
Section 3.3's residual sums).  On one GPU the exchange is a sum of the
slices' device buffers, standing in for the all-reduce of a multi-GPU run.

Against the whole-problem context the iterates agree to 2^-23 normwise per
iteration run (the sums over k are split across slices, so their rounding
differs), and against the FP64 oracle to the usual 1e-5; the penalty
decisions, the stopping test and the per-slice price parts agree."""
import numpy as np
import pytest

from gridgen import make_case, scale_case
from helpers import compare_states, rel_err
from oracle import Oracle, OracleOptions

pytestmark = pytest.mark.gpu

# Slices sum each device node's k-rows in FP32 per slice and add the slices'
# sums, the whole context sums all rows in FP32: the device inputs differ by
# about one FP32 rounding per iteration, which the nonexpansive iteration
# carries along without amplifying -- about 2^-23 relative per iteration.
SPLIT_RTOL = 2.0 ** -23


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2410_17203_gb300 import load_library
    load_library()


class Slices:
    def __init__(self, case, bounds, opts):
        from paper_2410_17203_gb300 import opf_create_slice, opf_slice_exchange, opf_slice_prime
        self.hs = [opf_create_slice(case, a, b, opts) for a, b in bounds]
        self.xs = [opf_slice_exchange(h) for h in self.hs]
        for h in self.hs:
            opf_slice_prime(h)
        self.exchange()

    def exchange(self):
        tot = self.xs[0].clone()
        for x in self.xs[1:]:
            tot += x
        for x in self.xs:
            x.copy_(tot)

    def iterate(self, n):
        from paper_2410_17203_gb300 import opf_slice_begin, opf_slice_finish, opf_slice_local
        for h in self.hs:
            opf_slice_begin(h, n)
        for _ in range(n):
            for h in self.hs:
                opf_slice_local(h)
            self.exchange()
            for h in self.hs:
                opf_slice_finish(h)

    def state(self):
        from paper_2410_17203_gb300 import opf_get_state
        parts = [opf_get_state(h) for h in self.hs]
        return {k: (parts[0][k] if k in ("p_dev", "inner") else np.concatenate([p[k] for p in parts], axis=0))
                for k in parts[0]}

    def close(self):
        from paper_2410_17203_gb300 import opf_destroy
        for h in self.hs:
            opf_destroy(h)


CASES = {
    "mixed_T24": (lambda: make_case(scale_case(150, 24, 6, seed=21)), [(0, 3), (3, 7)]),
    "three_slices": (lambda: make_case(scale_case(150, 24, 6, seed=21)), [(0, 1), (1, 4), (4, 7)]),
    "hvdc_scalar_T7": (lambda: make_case(scale_case(90, 7, 3, seed=22, fixed_frac=0.3, n_hvdc=2)), [(0, 2), (2, 4)]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_slices_match_the_whole_context_and_the_oracle(name):
    from paper_2410_17203_gb300 import Solver, opf_get_info, opf_residuals, opf_solution
    make, bounds = CASES[name]
    case = make()
    opts = dict(adapt_every=10, eps=0.0)
    sl = Slices(case, bounds, opts)
    whole = Solver(case, opts)
    try:
        for n in (25, 15):                       # two calls: the residuals at each call's end
            sl.iterate(n)
            whole.iterate(n)
        st, ref = sl.state(), whole.state()
        for k in ref:
            assert rel_err(st[k], ref[k]) <= SPLIT_RTOL * 40, (k, rel_err(st[k], ref[k]))
        o = Oracle(case, OracleOptions(**opts))
        o.iterate(40, stop=False)
        compare_states({k: v for k, v in st.items() if k != "inner"}, o)
        iw = whole.get_info()
        for h in sl.hs:
            i = opf_get_info(h)
            assert i["iterations"] == 40
            assert (i["rho_p"], i["rho_theta"]) == (iw["rho_p"], iw["rho_theta"])
            res = opf_residuals(h)
            np.testing.assert_allclose(res, whole.residuals(), rtol=1e-4)
        # prices: the slices' parts of -rho_p sum_k u_k add up to the whole
        N, T = case["n_nodes"], case["T"]
        parts = []
        for h in sl.hs:
            pr = np.zeros((N, T), np.float32)
            opf_solution(h, False, False, price=pr)
            parts.append(pr.astype(np.float64))
        assert rel_err(sum(parts), whole.solution()["price"]) <= 1e-6
    finally:
        sl.close()
        whole.close()


def test_slices_stop_together_at_the_tolerance():
    """Stopping test on the exchanged residuals: every slice stops at the
    same iteration, within a few stopping tests of the whole context, with
    the same objective and prices; a later call continues from the stopped
    state (a stopped slice keeps contributing its current sums) and stops
    again at the next test, as the whole context does."""
    from paper_2410_17203_gb300 import Solver, opf_get_info, opf_solution
    case = make_case("tiny")
    opts = dict(adapt_every=0, rho_theta=10.0, eps=1e-4)
    sl = Slices(case, [(0, 2), (2, 6)], opts)
    whole = Solver(case, opts)
    try:
        for _ in range(100):
            sl.iterate(500)
            if opf_get_info(sl.hs[0])["converged"]:
                break
        whole.iterate(50000)
        iw = whole.get_info()
        assert iw["converged"] == 1
        infos = [opf_get_info(h) for h in sl.hs]
        its = [i["iterations"] for i in infos]
        assert all(i["converged"] == 1 for i in infos) and all(i == its[0] for i in its)
        assert abs(its[0] - iw["iterations"]) <= 0.02 * iw["iterations"]

        def objective_and_price():
            N, T = case["n_nodes"], case["T"]
            obj, price = None, np.zeros((N, T))
            for h in sl.hs:
                pr = np.zeros((N, T), np.float32)
                o = opf_solution(h, False, True, price=pr)
                obj = o if obj is None else obj
                assert o == obj                      # devices are replicated: one objective
                price += pr
            return obj, price
        obj, price = objective_and_price()
        sol = whole.solution()
        assert obj == pytest.approx(sol["objective"], rel=1e-5)
        assert rel_err(price, sol["price"]) <= 1e-3
        sl.iterate(500)
        its2 = [opf_get_info(h)["iterations"] for h in sl.hs]
        assert all(i == its2[0] for i in its2) and its[0] < its2[0] <= its[0] + 500
        assert all(opf_get_info(h)["converged"] == 1 for h in sl.hs)
        assert objective_and_price()[0] == pytest.approx(obj, rel=1e-2)   # both pass the 1e-4 test
    finally:
        sl.close()
        whole.close()


def test_slices_continue_from_an_imported_state():
    """A warm start: each slice imports its block of a whole context's state,
    primes and exchanges, and continues like the whole context."""
    from paper_2410_17203_gb300 import Solver, opf_set_state, opf_slice_prime
    case = make_case(scale_case(150, 24, 6, seed=21))
    opts = dict(adapt_every=0, eps=0.0, rho_theta=5.0)
    whole = Solver(case, opts)
    sl = Slices(case, [(0, 4), (4, 7)], opts)
    try:
        whole.iterate(30)
        st = whole.state()
        for h, (a, b) in zip(sl.hs, [(0, 4), (4, 7)]):
            part = {k: (v if k in ("p_dev", "inner") else v[a:b]) for k, v in st.items()}
            opf_set_state(h, part)
            opf_slice_prime(h)
        sl.exchange()
        whole.set_state(st)
        sl.iterate(20)
        whole.iterate(20)
        got, ref = sl.state(), whole.state()
        for k in ref:
            assert rel_err(got[k], ref[k]) <= SPLIT_RTOL * 20, k
    finally:
        sl.close()
        whole.close()


@pytest.mark.slow
def test_benchmark_instance_as_four_slices():
    """The 10k workload (K = 50) split into four slices of 13, 13, 13 and 12
    contingencies, the launch configuration of a four-GPU benchmark run:
    after 20 iterations (two adaptations) every state array within the
    split-sum bound of the whole context, the same penalties and
    residuals."""
    from paper_2410_17203_gb300 import Solver, opf_get_info, opf_residuals
    case = make_case("10k")
    opts = dict(adapt_every=10, eps=0.0)
    blocks = np.array_split(np.arange(51), 4)
    sl = Slices(case, [(int(b[0]), int(b[-1]) + 1) for b in blocks], opts)
    whole = Solver(case, opts)
    try:
        sl.iterate(20)
        whole.iterate(20)
        st, ref = sl.state(), whole.state()
        for k in ref:
            assert rel_err(st[k], ref[k]) <= SPLIT_RTOL * 20, (k, rel_err(st[k], ref[k]))
        iw = whole.get_info()
        for h in sl.hs:
            i = opf_get_info(h)
            assert (i["rho_p"], i["rho_theta"], i["iterations"]) == (iw["rho_p"], iw["rho_theta"], 20)
            np.testing.assert_allclose(opf_residuals(h), whole.residuals(), rtol=1e-4)
    finally:
        sl.close()
        whole.close()


@pytest.mark.parametrize("K, bounds", [(0, [(0, 1)]), (2, [(0, 1), (1, 2), (2, 3)])])
def test_single_contingency_slices(K, bounds):
    """Degenerate blocks: the base case alone as one slice (K = 0), and one
    contingency per slice."""
    from paper_2410_17203_gb300 import Solver
    case = make_case(scale_case(60, 8, K, seed=41))
    opts = dict(adapt_every=10, eps=0.0)
    sl = Slices(case, bounds, opts)
    whole = Solver(case, opts)
    try:
        sl.iterate(30)
        whole.iterate(30)
        st, ref = sl.state(), whole.state()
        for k in ref:
            assert rel_err(st[k], ref[k]) <= SPLIT_RTOL * 30, k
    finally:
        sl.close()
        whole.close()


def test_slice_refuses_whole_context_calls():
    from paper_2410_17203_gb300 import OpfError, opf_batch_create, opf_create_slice, opf_destroy, opf_iterate
    case = make_case("tiny")
    h = opf_create_slice(case, 0, 3)
    try:
        with pytest.raises(OpfError) as e:
            opf_iterate(h, 5)
        assert e.value.status == 6                     # OPF_ESTATE
        with pytest.raises(OpfError):
            opf_batch_create([h])
    finally:
        opf_destroy(h)
