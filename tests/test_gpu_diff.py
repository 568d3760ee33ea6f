"""Parity of the unrolled-iteration gradients (include/opf_diff.h, Section 4.4
and Section 5.5) against the PyTorch FP64 autograd reference oracle/unrolled.py.

The device path runs in FP32.  Every step of the iteration is nonexpansive
up to the penalty ratios, so the rounding of K steps grows roughly linearly
with K (about 1e-6 relative per step); the gradients are compared normwise
at 2e-3 for K <= 60 and the cost at 1e-4 relative.  Clipping decisions are
taken on FP32 values on the device and FP64 values in the reference; the
seeded cases here have no bound ties at that precision (a tie would show as a
single large element, which the normwise test would report)."""
import numpy as np
import pytest
import torch

from gridgen import make_case, scale_case
from oracle.unrolled import Unrolled

pytestmark = pytest.mark.gpu

GRAD_RTOL = 2e-3
COST_RTOL = 1e-4


def _lib():
    from paper_2410_17203_gb300 import binding
    return binding


def _reference(case, K, rho_p, rho_theta):
    ur = Unrolled(case, rho_p=rho_p, rho_theta=rho_theta)
    prm = ur.params()
    f, _ = ur.run(prm, K)
    f.backward()
    return float(f.detach()), {k: v.grad.numpy() for k, v in prm.items()}


def _normwise(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0)


def _check(case, K, rho_p=10.0, rho_theta=20.0, ckpt=8):
    b = _lib()
    f_ref, g_ref = _reference(case, K, rho_p, rho_theta)
    d = b.UnrolledCost(case, rho_p=rho_p, rho_theta=rho_theta, checkpoint_every=ckpt)
    try:
        f, g = d.cost_grad(K)
    finally:
        d.close()
    assert f == pytest.approx(f_ref, rel=COST_RTOL)
    for k in ("load_p", "gen_pmax", "line_u"):
        assert g[k].shape == g_ref[k].shape
        assert _normwise(g[k], g_ref[k]) <= GRAD_RTOL, (k, _normwise(g[k], g_ref[k]))
    return g_ref


def test_small_case_matches_autograd():
    case = make_case(scale_case(40, 3, 2, seed=5, ramp=False, stor_per_node=0.0, fixed_frac=0.3))
    g = _check(case, 40)
    # at these penalties the case exercises every gradient path: fixed and
    # curtailable loads, generators at their capacity, lines at their limit
    assert np.count_nonzero(g["gen_pmax"]) > 0 and np.count_nonzero(g["line_u"]) > 0


def test_several_tiles_and_contingencies():
    case = make_case(scale_case(600, 5, 6, seed=11, ramp=False, stor_per_node=0.0, fixed_frac=0.2))
    _check(case, 60, rho_p=1.0, rho_theta=5.0, ckpt=7)


def test_base_case_only_and_single_step():
    case = make_case(scale_case(50, 1, 0, seed=3, ramp=True, stor_per_node=0.0, fixed_frac=0.5))
    _check(case, 1)
    _check(case, 25, rho_p=50.0, rho_theta=100.0, ckpt=25)


def test_checkpointing_is_exact():
    """Recomputed segments repeat the forward pass bit for bit, so the
    gradients do not depend on the checkpoint spacing, nor on whether the
    reverse pass reads the forward's record of clipped values (and then no
    state, so nothing is recomputed) or recomputes them (record limit 0; a
    limit too small for this call)."""
    b = _lib()
    case = make_case(scale_case(120, 4, 3, seed=8, ramp=True, stor_per_node=0.05, fixed_frac=0.3, n_hvdc=2))
    outs = []
    for ckpt, limit in ((1, None), (5, None), (64, None), (1, 0), (5, 0), (5, 1000)):
        d = b.UnrolledCost(case, rho_p=10.0, rho_theta=20.0, checkpoint_every=ckpt)
        try:
            if limit is not None:
                d.set_record_limit(limit)
            outs.append(d.cost_grad(37))
        finally:
            d.close()
    for f, g in outs[1:]:
        assert f == outs[0][0]
        for k in g:
            np.testing.assert_array_equal(g[k], outs[0][1][k])
    # the same context switching between the two
    d = b.UnrolledCost(case, rho_p=10.0, rho_theta=20.0, checkpoint_every=5)
    try:
        d.set_record_limit(0)
        f0, g0 = d.cost_grad(23)
        d.set_record_limit(1 << 30)
        f1, g1 = d.cost_grad(23)
        with pytest.raises(b.OpfError):
            d.set_record_limit(-1)
    finally:
        d.close()
    assert f0 == f1
    for k in g0:
        np.testing.assert_array_equal(g0[k], g1[k])


def test_data_arguments_replace_the_case_data():
    """Passing changed data equals differentiating the changed case."""
    b = _lib()
    case = make_case(scale_case(60, 2, 2, seed=4, ramp=False, stor_per_node=0.0, fixed_frac=0.3))
    rng = np.random.default_rng(1)
    lp = np.asarray(case["load_p"]) * (1 + 0.2 * rng.random(np.shape(case["load_p"])))
    pm = np.asarray(case["gen_pmax"]) * 0.8
    lu = np.asarray(case["line_u"]) * 0.7
    changed = dict(case, load_p=lp, gen_pmax=pm, line_u=lu)
    d = b.UnrolledCost(case, rho_p=10.0, rho_theta=20.0)
    try:
        f, g = d.cost_grad(30, load_p=lp, gen_pmax=pm, line_u=lu)
        f0, g0 = d.cost_grad(30)
        f_none, g_none = d.cost_grad(30, grads=False)
    finally:
        d.close()
    f_ref, g_ref = _reference(changed, 30, 10.0, 20.0)
    assert f == pytest.approx(f_ref, rel=COST_RTOL)
    for k in g:
        assert _normwise(g[k], g_ref[k]) <= GRAD_RTOL
    assert f_none == f0 and g_none is None
    assert f0 != f


def test_inner_admm_devices_match_autograd():
    """Ramp-limited generators and batteries: the reverse pass runs through
    the ten inner ADMM iterations of every outer iteration (Appendix D)."""
    case = make_case(scale_case(40, 6, 2, seed=7, ramp=True, stor_per_node=0.1, fixed_frac=0.3))
    _check(case, 40, ckpt=9)
    case = make_case(scale_case(30, 1, 3, seed=9, ramp=True, stor_per_node=0.2, fixed_frac=0.3))
    _check(case, 30, ckpt=4)                       # T = 1: batteries only


@pytest.mark.parametrize("T", [31, 32, 70, 127, 130])
def test_inner_admm_horizons_match_autograd(T):
    """The inner ADMM from registers at one to four steps per lane (the chunk
    boundaries of T + 1 = 32, 33 and 128 states of charge), and beyond 127
    steps through the shared-memory path with the system's inverse."""
    case = make_case(scale_case(12, T, 1, seed=40 + T, ramp=True, stor_per_node=0.3, fixed_frac=0.3))
    _check(case, 15, ckpt=4)


def test_hvdc_links_match_autograd():
    case = make_case(scale_case(40, 6, 2, seed=7, ramp=True, stor_per_node=0.1, fixed_frac=0.3, n_hvdc=2))
    _check(case, 40, ckpt=9)


def test_inner_admm_devices_several_tiles():
    case = make_case(scale_case(300, 24, 4, seed=12, ramp=True, stor_per_node=0.05, fixed_frac=0.2))
    _check(case, 40, rho_p=5.0, rho_theta=10.0, ckpt=6)


def test_rejects_invalid_data():
    b = _lib()
    bad = make_case(scale_case(40, 3, 1, seed=2, ramp=False, stor_per_node=0.2))
    bad["stor_eff"] = np.zeros(len(bad["stor_node"]))
    with pytest.raises(b.OpfError):
        b.UnrolledCost(bad)
    with pytest.raises(b.OpfError):
        b.UnrolledCost(make_case(scale_case(40, 1, 1, seed=2, ramp=False, stor_per_node=0.0)), rho_p=0.0)


def test_torch_tensors_are_accepted():
    b = _lib()
    case = make_case(scale_case(40, 2, 1, seed=6, ramp=False, stor_per_node=0.0, fixed_frac=0.3))
    d = b.UnrolledCost(case, rho_p=10.0, rho_theta=20.0)
    try:
        f1, g1 = d.cost_grad(10, load_p=torch.tensor(np.asarray(case["load_p"])))
        f2, g2 = d.cost_grad(10)
    finally:
        d.close()
    assert f1 == f2
    np.testing.assert_array_equal(g1["load_p"], g2["load_p"])


def test_autograd_function():
    """unrolled_cost plugs the device gradients into torch.autograd; a
    gradient step on the capacities of the cheapest generators lowers the
    cost (the use Section 5.6 makes of these derivatives)."""
    b = _lib()
    case = make_case(scale_case(60, 2, 2, seed=4, ramp=False, stor_per_node=0.0, fixed_frac=0.3))
    d = b.UnrolledCost(case, rho_p=10.0, rho_theta=20.0)
    try:
        lp = torch.tensor(np.asarray(case["load_p"]), dtype=torch.float64, requires_grad=True)
        pm = torch.tensor(np.asarray(case["gen_pmax"]), dtype=torch.float64, requires_grad=True)
        lu = torch.tensor(np.asarray(case["line_u"]), dtype=torch.float64, requires_grad=True)
        f = b.unrolled_cost(d, 30, lp, pm, lu)
        (2.0 * f).backward()
        f_ref, g_ref = d.cost_grad(30)
        assert float(f.detach()) == f_ref
        np.testing.assert_allclose(pm.grad.numpy(), 2.0 * g_ref["gen_pmax"], rtol=1e-6)
        np.testing.assert_allclose(lp.grad.numpy(), 2.0 * g_ref["load_p"], rtol=1e-6)
        np.testing.assert_allclose(lu.grad.numpy(), 2.0 * g_ref["line_u"], rtol=1e-6)
        with torch.no_grad():
            pm2 = pm - 1e-3 * pm.grad / max(1.0, float(pm.grad.abs().max()))
        f2 = b.unrolled_cost(d, 30, lp.detach(), pm2, lu.detach())
        assert float(f2) < float(f.detach())
    finally:
        d.close()


def test_device_tensors_match_host_arrays_and_calls_repeat():
    """opf_diff_cost_grad_on with device pointers returns what the host-array
    entry returns, bit for bit (the same kernels on the same data); calls of
    different lengths reuse the context's buffers and repeat exactly; the
    autograd function keeps CUDA tensors on the device."""
    b = _lib()
    case = make_case(scale_case(80, 6, 3, seed=12, stor_per_node=0.1))
    d = b.UnrolledCost(case, rho_p=2.0, rho_theta=5.0, checkpoint_every=7)
    try:
        rng = np.random.default_rng(3)
        lp = np.asarray(case["load_p"]) * rng.uniform(0.9, 1.1, size=np.shape(case["load_p"]))
        pm = np.asarray(case["gen_pmax"]) * rng.uniform(0.9, 1.1, size=np.shape(case["gen_pmax"]))
        lu = np.asarray(case["line_u"]) * rng.uniform(0.9, 1.1, size=np.shape(case["line_u"]))
        f_h, g_h = d.cost_grad(40, lp, pm, lu)
        dv = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in (lp, pm, lu)]
        f_d, g_d = d.cost_grad_device(40, *dv)
        assert f_d == f_h
        for k in g_h:
            np.testing.assert_array_equal(g_d[k].cpu().numpy(), g_h[k], err_msg=k)
        f_short, _ = d.cost_grad(13, lp, pm, lu)         # a shorter call in between
        f_again, g_again = d.cost_grad(40, lp, pm, lu)
        assert f_again == f_h and f_short != f_h
        for k in g_h:
            np.testing.assert_array_equal(g_again[k], g_h[k], err_msg=k)
        xs = [x.clone().requires_grad_(True) for x in dv]
        f = b.unrolled_cost(d, 40, *xs)
        assert f.is_cuda and float(f.detach()) == float(np.float32(f_h))   # a float32 tensor
        f.backward()
        for x, k in zip(xs, ("load_p", "gen_pmax", "line_u")):
            assert x.grad.is_cuda
            np.testing.assert_array_equal(x.grad.cpu().numpy(), g_h[k], err_msg=k)
    finally:
        d.close()


def test_gradients_approach_the_duals():
    """Section 5.5: with more unrolled iterations the derivatives approach
    the sensitivities of the optimal cost -- the nodal price for a fixed load
    and (2 a pmax + b) - price for a generator at its capacity.  The
    converged prices come from the FP64 oracle run to its fixed point."""
    from oracle import Oracle, OracleOptions
    b = _lib()
    case = make_case("tiny")                       # fixed loads, T = 1
    rp, rt = 10.0, 100.0
    o = Oracle(case, OracleOptions(adapt_every=0, rho_p=rp, rho_theta=rt, eps=0.0))
    o.iterate(30000, stop=False)
    lam = o.prices()[:, 0]
    want = lam[np.asarray(case["load_node"])]
    gn = np.asarray(case["gen_node"])
    pg = o.dev_p()[:len(gn), 0]
    pmax = np.asarray(case["gen_pmax"])[:, 0]
    mu = lam[gn] - (2 * np.asarray(case["gen_a"]) * pg + np.asarray(case["gen_b"]))
    at_cap = np.flatnonzero((mu > 1.0) & (np.abs(pg - pmax) < 1e-6))
    assert at_cap.size >= 1
    d = b.UnrolledCost(case, rho_p=rp, rho_theta=rt, checkpoint_every=200)
    try:
        errs = []
        for K in (3000, 24000):
            _, g = d.cost_grad(K)
            errs.append(np.linalg.norm(g["load_p"][:, 0] - want) / np.linalg.norm(want))
        cap = g["gen_pmax"][at_cap, 0]
    finally:
        d.close()
    assert errs[1] < 0.02 and errs[1] < 0.25 * errs[0], errs
    np.testing.assert_allclose(cap, -mu[at_cap], rtol=0.1)
