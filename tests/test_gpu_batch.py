"""Batched iteration (one CUDA graph over independent instances) gives the
same iterates as iterating each instance alone, and keeps converged
instances stopped while the others go on."""
import numpy as np
import pytest

from gridgen import make_case, scale_case
from helpers import hang_triangle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2410_17203_gb300 import load_library
    load_library()


def _cases():
    return [make_case("tiny"),
            make_case(scale_case(150, 24, 6, seed=21)),
            make_case(scale_case(90, 7, 3, seed=22, fixed_frac=0.3)),
            make_case(scale_case(70, 8, 0, seed=23, fixed_frac=0.5, stor_per_node=0.0)),
            make_case(scale_case(80, 12, 2, seed=27, n_hvdc=3)),
            hang_triangle(make_case(scale_case(40, 5, 1, seed=28)), node=3),
            # a horizon above 128 steps: inner-ADMM state in global memory
            make_case(scale_case(30, 150, 1, seed=30, stor_per_node=0.1, fixed_frac=0.3))]


def test_batch_iterates_equal_single_instance_iterates():
    from paper_2410_17203_gb300 import (Solver, opf_batch_create, opf_batch_destroy,
                                        opf_batch_iterate)
    opts = dict(adapt_every=10, eps=0.0)
    batch_solvers = [Solver(c, opts) for c in _cases()]
    single = [Solver(c, opts) for c in _cases()]
    b = opf_batch_create([s.h for s in batch_solvers])
    try:
        for n in (3, 16, 18):        # graphs of 1 and 16 iterations, and a mix
            opf_batch_iterate(b, n)
        for s in single:
            s.iterate(37)
        for sb, ss in zip(batch_solvers, single):
            a, c = sb.state(), ss.state()
            for k in a:
                np.testing.assert_array_equal(a[k], c[k], err_msg=k)
            assert sb.get_info()["iterations"] == 37
    finally:
        opf_batch_destroy(b)
        for s in batch_solvers + single:
            s.close()


def test_mixed_horizons_equal_single_instance_iterates():
    """Horizons of 1, 24, 48, 96 and 150 steps in one batch: the inner ADMM
    runs from registers at every horizon up to 127 steps, each with its own
    chunk of steps per lane, in a kernel sized for the longest (and in
    shared memory at 150 steps), and still repeats the single-instance
    iterates bit for bit."""
    from paper_2410_17203_gb300 import (Solver, opf_batch_create, opf_batch_destroy,
                                        opf_batch_iterate)
    specs = [scale_case(100, 1, 3, seed=23), scale_case(150, 24, 6, seed=21), scale_case(120, 48, 4, seed=22),
             scale_case(120, 96, 4, seed=24), scale_case(30, 150, 1, seed=30, stor_per_node=0.1)]
    cases = [make_case(sp) for sp in specs]
    opts = dict(adapt_every=10, eps=0.0)
    batch_solvers = [Solver(c, opts) for c in cases]
    single = [Solver(c, opts) for c in cases]
    b = opf_batch_create([s.h for s in batch_solvers])
    try:
        opf_batch_iterate(b, 23)
        for s in single:
            s.iterate(23)
        for sb, ss, sp in zip(batch_solvers, single, specs):
            a, c = sb.state(), ss.state()
            for k in a:
                np.testing.assert_array_equal(a[k], c[k], err_msg=f"T={sp['T']} {k}")
    finally:
        opf_batch_destroy(b)
        for s in batch_solvers + single:
            s.close()


def test_compaction_keeps_iterates_and_drops_stopped_instances():
    """opf_batch_compact after some instances have stopped (here: converged
    early at a loose tolerance): the schedule keeps the running ones, whose
    iterates stay bit for bit those of single-instance runs (layout, CTA
    split and residual partial sums unchanged), and the stopped ones keep
    their state."""
    from paper_2410_17203_gb300 import (Solver, opf_batch_autotune, opf_batch_compact, opf_batch_create,
                                        opf_batch_destroy, opf_batch_iterate, opf_batch_stopped)
    cases = [make_case("tiny"), make_case(scale_case(150, 24, 6, seed=21)), make_case(scale_case(90, 7, 3, seed=22)),
             make_case(scale_case(80, 12, 2, seed=27, n_hvdc=3))]
    # the tiny case converges within the first 300 iterations at this tolerance
    opts = [dict(adapt_every=10, eps=1e-2, rho_theta=10.0)] + [dict(adapt_every=10, eps=0.0)] * 3
    bs = [Solver(c, o) for c, o in zip(cases, opts)]
    ss = [Solver(c, o) for c, o in zip(cases, opts)]
    b = opf_batch_create([s.h for s in bs])
    try:
        opf_batch_autotune(b, steps=3)
        assert opf_batch_compact(b) == 4          # nothing stopped yet
        opf_batch_iterate(b, 300)
        assert opf_batch_stopped(b)[0] == 1
        assert opf_batch_compact(b) == 3
        frozen = bs[0].state()
        opf_batch_iterate(b, 37)
        for s in ss:
            s.iterate(337)
        np.testing.assert_equal(bs[0].state(), frozen)
        stopped_at = bs[0].get_info()["iterations"]
        assert stopped_at == ss[0].get_info()["iterations"] and stopped_at < 300
        for sb, s1 in zip(bs[1:], ss[1:]):
            a, c = sb.state(), s1.state()
            for k in a:
                np.testing.assert_array_equal(a[k], c[k], err_msg=k)
            assert sb.get_info()["iterations"] == 337
            np.testing.assert_array_equal(sb.residuals(), s1.residuals())
    finally:
        opf_batch_destroy(b)
        for s in bs + ss:
            s.close()


def test_compaction_when_every_instance_has_stopped_and_after_autotune():
    """A batch whose instances have all stopped compacts to an empty schedule
    (later steps change nothing); opf_batch_autotune schedules every
    instance again."""
    from paper_2410_17203_gb300 import (Solver, opf_batch_autotune, opf_batch_compact, opf_batch_create,
                                        opf_batch_destroy, opf_batch_iterate, opf_batch_stopped)
    opts = dict(adapt_every=10, eps=1e-2, rho_theta=10.0)
    solvers = [Solver(make_case("tiny"), opts), Solver(make_case("tiny"), dict(opts, rho_theta=5.0))]
    b = opf_batch_create([s.h for s in solvers])
    try:
        opf_batch_iterate(b, 600)
        assert opf_batch_stopped(b)[0] == 2
        assert opf_batch_compact(b) == 0
        before = [s.state() for s in solvers]
        its = [s.get_info()["iterations"] for s in solvers]
        opf_batch_iterate(b, 50)
        for s, st, it in zip(solvers, before, its):
            np.testing.assert_equal(s.state(), st)
            assert s.get_info()["iterations"] == it
        opf_batch_autotune(b, steps=2)          # leaves the stopped instances as they are
        assert opf_batch_compact(b) == 0
    finally:
        opf_batch_destroy(b)
        for s in solvers:
            s.close()


def test_converged_instances_stay_stopped():
    from paper_2410_17203_gb300 import (Solver, opf_batch_converged, opf_batch_create,
                                        opf_batch_destroy, opf_batch_iterate)
    # the same instance at two fixed penalties: they converge at different
    # iterations, and the first must not move while the second goes on
    base = dict(adapt_every=0, eps=1e-4)
    solvers = [Solver(make_case("tiny"), dict(base, rho_theta=10.0)),
               Solver(make_case("tiny"), dict(base, rho_theta=5.0))]
    b = opf_batch_create([s.h for s in solvers])
    try:
        for _ in range(400):
            opf_batch_iterate(b, 100)
            if opf_batch_converged(b) == len(solvers):
                break
        assert opf_batch_converged(b) == len(solvers)
        its = [s.get_info()["iterations"] for s in solvers]
        assert its[0] != its[1]
        opf_batch_iterate(b, 50)
        assert [s.get_info()["iterations"] for s in solvers] == its
        for s in solvers:
            res = s.residuals()
            assert max(res[0], res[1]) <= s.get_info()["tolerance"]
    finally:
        opf_batch_destroy(b)
        for s in solvers:
            s.close()


def test_batch_rejects_bad_arguments():
    from paper_2410_17203_gb300 import OpfError, Solver, opf_batch_create
    s = Solver(make_case("tiny"), dict(eps=0.0))
    try:
        with pytest.raises(OpfError):
            opf_batch_create([s.h, s.h])
    finally:
        s.close()


def test_autotune_keeps_iterates_and_the_chosen_layout_is_exact():
    """The autotuner restores the instances' states, and whichever layout it
    keeps, later batch iterates equal single-instance iterates bit for bit."""
    from paper_2410_17203_gb300 import (BATCH_LAYOUTS, Solver, opf_batch_autotune, opf_batch_create,
                                        opf_batch_destroy, opf_batch_iterate)
    opts = dict(adapt_every=10, eps=0.0)
    batch_solvers = [Solver(c, opts) for c in _cases()]
    single = [Solver(c, opts) for c in _cases()]
    b = opf_batch_create([s.h for s in batch_solvers])
    try:
        opf_batch_iterate(b, 5)
        before = [s.state() for s in batch_solvers]
        choice, ms = opf_batch_autotune(b, steps=8)
        assert 0 <= choice < len(BATCH_LAYOUTS) and len(ms) == len(BATCH_LAYOUTS)
        assert all(m > 0 for m in ms) and ms[choice] == min(ms)
        for s, st in zip(batch_solvers, before):
            a = s.state()
            for k in a:
                np.testing.assert_array_equal(a[k], st[k], err_msg=k)
            assert s.get_info()["iterations"] == 5
        opf_batch_iterate(b, 20)
        for s in single:
            s.iterate(25)
        for sb, ss in zip(batch_solvers, single):
            a, c = sb.state(), ss.state()
            for k in a:
                np.testing.assert_array_equal(a[k], c[k], err_msg=k)
    finally:
        opf_batch_destroy(b)
        for s in batch_solvers + single:
            s.close()


def test_over_relaxed_batch_equals_single_and_mixing_is_rejected():
    from paper_2410_17203_gb300 import (OpfError, Solver, opf_batch_create, opf_batch_destroy,
                                        opf_batch_iterate)
    opts = dict(adapt_every=10, eps=0.0, alpha=1.5)
    batch_solvers = [Solver(c, opts) for c in _cases()]
    single = [Solver(c, opts) for c in _cases()]
    b = opf_batch_create([s.h for s in batch_solvers])
    try:
        opf_batch_iterate(b, 21)
        for s in single:
            s.iterate(21)
        for sb, ss in zip(batch_solvers, single):
            a, c = sb.state(), ss.state()
            for k in a:
                np.testing.assert_array_equal(a[k], c[k], err_msg=k)
        plain = Solver(make_case("tiny"), dict(adapt_every=10, eps=0.0))
        try:
            with pytest.raises(OpfError):
                opf_batch_create([batch_solvers[0].h, plain.h])
        finally:
            plain.close()
    finally:
        opf_batch_destroy(b)
        for s in batch_solvers + single:
            s.close()


@pytest.mark.parametrize("alpha", [1.0, 1.5])
def test_batch_iterates_match_the_oracle(alpha):
    """Every instance of a batch (uneven sizes, T from 1 to 150, outages,
    HVDC links, device-free nodes), after 37 batch iterations in three calls
    (graphs of 1 and 16 iterations) with the adaptive penalty, against the
    FP64 oracle run on that instance alone: normwise 1e-5 per state array,
    the same penalties."""
    from helpers import compare_states
    from oracle import Oracle, OracleOptions
    from paper_2410_17203_gb300 import Solver, opf_batch_create, opf_batch_destroy, opf_batch_iterate
    opts = dict(adapt_every=10, eps=0.0, alpha=alpha)
    cases = _cases()
    solvers = [Solver(c, opts) for c in cases]
    b = opf_batch_create([s.h for s in solvers])
    try:
        for n in (3, 16, 18):
            opf_batch_iterate(b, n)
        for s, c in zip(solvers, cases):
            o = Oracle(c, OracleOptions(**opts))
            o.iterate(37, stop=False)
            compare_states(s.state(), o)
            info = s.get_info()
            assert (info["rho_p"], info["rho_theta"]) == pytest.approx((o.rho_p, o.rho_th), rel=1e-12)
    finally:
        opf_batch_destroy(b)
        for s in solvers:
            s.close()


def test_batched_workload_instances_match_the_oracle():
    """Instances drawn by the batched workload's recipe (buses log-uniform in
    [100, 5000], T in {1, 24, 48}, 0..20 outages; the smaller ones, so that
    the oracle finishes in seconds), batched after autotuning, against the
    oracle after 30 iterations."""
    from helpers import compare_states
    from oracle import Oracle, OracleOptions
    from paper_2410_17203_gb300 import (Solver, opf_batch_autotune, opf_batch_create, opf_batch_destroy,
                                        opf_batch_iterate)
    rng = np.random.default_rng(3)
    specs = []
    for i in range(40):
        nb = int(round(float(np.exp(rng.uniform(np.log(100), np.log(5000))))))
        T = int(rng.choice([1, 24, 48]))
        K = int(rng.integers(0, 21))
        if nb * T * (K + 1) <= 200000:
            specs.append(scale_case(nb, T, K, seed=1000 + i, lines_per_node=1.5))
    assert len(specs) >= 4
    cases = [make_case(sp) for sp in specs]
    opts = dict(adapt_every=10, eps=0.0)
    solvers = [Solver(c, opts) for c in cases]
    b = opf_batch_create([s.h for s in solvers])
    try:
        opf_batch_autotune(b, steps=4)
        opf_batch_iterate(b, 30)
        for s, c in zip(solvers, cases):
            o = Oracle(c, OracleOptions(**opts))
            o.iterate(30, stop=False)
            compare_states(s.state(), o)
    finally:
        opf_batch_destroy(b)
        for s in solvers:
            s.close()
