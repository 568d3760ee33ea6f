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


def test_too_large_network_is_rejected_before_device_work():
    from paper_2410_17203_gb300 import OpfError, Solver, opf_price_noalloc
    from paper_2410_17203_gb300.binding import OPF_PRICE_SCRATCH_FLOATS
    case = make_case(scale_case(1200, 900, 0, seed=5, stor_per_node=0.0))
    assert case["n_nodes"] * case["T"] > OPF_PRICE_SCRATCH_FLOATS
    s = Solver(case, dict(eps=0.0))
    try:
        with pytest.raises(OpfError) as e:
            opf_price_noalloc(s.h, np.zeros((case["n_nodes"], case["T"]), np.float32))
        assert e.value.status == 1
        assert "OPF_PRICE_SCRATCH_FLOATS" in str(e.value)
    finally:
        s.close()
