"""opf_price_noalloc: the price export staged through the library's fixed
device array, against opf_solution's price (which stages through a per-call
device buffer), on two consecutive calls with iterations in between.

The file name sorts last so that the fixed array has already been used by
the other tests' contexts when this runs in the full suite; it also passes
alone."""
import numpy as np
import pytest

from gridgen import make_case, scale_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2410_17203_gb300 import load_library
    load_library()


def _price_via_solution(s):
    info = s.get_info()
    out = np.zeros((info["N"], info["T"]), np.float32)
    from paper_2410_17203_gb300 import opf_solution
    opf_solution(s.h, on_device=False, objective=False, price=out)
    return out


@pytest.mark.parametrize("case", [
    lambda: make_case("tiny"),
    lambda: make_case(scale_case(150, 24, 6, seed=21)),
    lambda: make_case(scale_case(90, 7, 3, seed=22, fixed_frac=0.3)),
])
def test_two_consecutive_calls_match_solution_price(case):
    from paper_2410_17203_gb300 import Solver, opf_price_noalloc
    s = Solver(case(), dict(adapt_every=10, eps=0.0))
    try:
        s.iterate(13)
        a = opf_price_noalloc(s.h)
        np.testing.assert_array_equal(a, _price_via_solution(s))
        assert np.isfinite(a).all() and np.abs(a).max() > 0
        s.iterate(21)
        b = np.full_like(a, np.nan)
        opf_price_noalloc(s.h, b)
        np.testing.assert_array_equal(b, _price_via_solution(s))
        assert not np.array_equal(a, b)
    finally:
        s.close()


def test_two_contexts_use_the_same_array_one_after_the_other():
    from paper_2410_17203_gb300 import Solver, opf_price_noalloc
    s1 = Solver(make_case(scale_case(150, 24, 6, seed=21)), dict(eps=0.0))
    s2 = Solver(make_case("tiny"), dict(eps=0.0))
    try:
        s1.iterate(9)
        s2.iterate(9)
        p1 = opf_price_noalloc(s1.h)
        p2 = opf_price_noalloc(s2.h)
        np.testing.assert_array_equal(p1, _price_via_solution(s1))
        np.testing.assert_array_equal(p2, _price_via_solution(s2))
    finally:
        s1.close()
        s2.close()


def test_largest_network_is_exported_in_full():
    """N * T exactly OPF_PRICE_SCRATCH_FLOATS (1024 buses, T = 1024): every
    element of the array is staged and copied out."""
    from paper_2410_17203_gb300 import Solver, opf_price_noalloc
    from paper_2410_17203_gb300.binding import OPF_PRICE_SCRATCH_FLOATS
    case = make_case(scale_case(1024, 1024, 0, seed=6, stor_per_node=0.0))
    assert case["n_nodes"] * case["T"] == OPF_PRICE_SCRATCH_FLOATS
    s = Solver(case, dict(eps=0.0))
    try:
        s.iterate(7)
        out = np.full((case["n_nodes"], case["T"]), np.nan, np.float32)
        opf_price_noalloc(s.h, out)
        ref = _price_via_solution(s)
        np.testing.assert_array_equal(out, ref)
        assert np.isfinite(out).all() and np.abs(out).max() > 0
    finally:
        s.close()


def test_network_above_the_limit_is_rejected_and_the_context_still_works():
    """N * T one row of T above the capacity (1025 buses, T = 1024): the call
    fails with OPF_EINVAL, leaves the output untouched, and the context's
    iterate and later calls are unaffected."""
    from paper_2410_17203_gb300 import OpfError, Solver, opf_price_noalloc
    from paper_2410_17203_gb300.binding import OPF_PRICE_SCRATCH_FLOATS
    case = make_case(scale_case(1025, 1024, 0, seed=5, stor_per_node=0.0))
    assert case["n_nodes"] * case["T"] == OPF_PRICE_SCRATCH_FLOATS + 1024
    s = Solver(case, dict(eps=0.0))
    try:
        s.iterate(3)
        before = s.state()
        out = np.full((case["n_nodes"], case["T"]), 7.0, np.float32)
        with pytest.raises(OpfError) as e:
            opf_price_noalloc(s.h, out)
        assert e.value.status == 1
        assert "OPF_PRICE_SCRATCH_FLOATS" in str(e.value)
        assert np.all(out == 7.0)
        assert s.get_info()["iterations"] == 3
        after = s.state()
        for k in before:
            np.testing.assert_array_equal(before[k], after[k], err_msg=k)
        price = _price_via_solution(s)
        assert np.isfinite(price).all()
        s.iterate(2)
        assert s.get_info()["iterations"] == 5
    finally:
        s.close()
