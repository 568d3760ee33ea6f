"""The seeded input generators follow their stated recipe (CPU only).

The generators hold none of the method's arithmetic; these checks pin the
workload shapes (buses, lines, devices, horizon, contingencies), the value
ranges of each draw, determinism per seed, and the two structural claims the
recipe makes: every outage keeps the grid connected, and the flow limits admit
the capacity-proportional dispatch in every contingency (so the instances are
feasible).  The connectivity and flow checks use dense linear algebra written
here, not the generator's sparse helpers."""
import numpy as np
import pytest

from gridgen import case_dims, make_case, scale_case
from gridgen.cases import VOLL


@pytest.mark.parametrize("name, want", [
    ("tiny", dict(N=30, L=40, G=6, D=20, B=0, T=1, K=5, J=106)),
    ("2k", dict(N=2000, L=3200, G=500, D=1500, B=100, T=24, K=20, J=8500)),
    ("10k", dict(N=10000, L=15000, G=2500, D=7500, B=500, T=96, K=50, J=40500)),
])
def test_named_workload_sizes(name, want):
    d = case_dims(make_case(name))
    assert {k: d[k] for k in want} == want
    assert d["S"] == want["G"] + want["D"] + want["B"]


def test_generation_is_deterministic_per_seed():
    a, b = make_case("2k"), make_case("2k")
    for k, v in a.items():
        np.testing.assert_array_equal(np.asarray(v), np.asarray(b[k]), err_msg=k)
    c = make_case("2k", seed=7)
    assert not np.array_equal(a["load_p"], c["load_p"])


def _laplacian(n, frm, to, b):
    Bm = np.zeros((n, n))
    np.add.at(Bm, (frm, frm), b)
    np.add.at(Bm, (to, to), b)
    np.add.at(Bm, (frm, to), -b)
    np.add.at(Bm, (to, frm), -b)
    return Bm


def _dense_flows(case, inj, drop=None):
    """DC power flow: angles from the reduced Laplacian (node 0 as reference),
    flow b (theta_from - theta_to) on every line that is in service."""
    n = case["n_nodes"]
    frm, to, b = (np.asarray(case[k]) for k in ("line_from", "line_to", "line_b"))
    b = b.copy()
    if drop is not None:
        b[drop] = 0.0
    Bm = _laplacian(n, frm, to, b)
    th = np.zeros((n, inj.shape[1]))
    th[1:] = np.linalg.solve(Bm[1:, 1:], inj[1:])
    return b[:, None] * (th[frm] - th[to])


@pytest.mark.parametrize("case", [make_case("tiny"), make_case(scale_case(300, 24, 8, seed=5)),
                                  make_case(scale_case(120, 1, 12, seed=6, topology="random_tree"))],
                         ids=["tiny", "geometric_300", "tree_120"])
def test_outages_are_distinct_and_keep_the_grid_connected(case):
    n = case["n_nodes"]
    frm, to, b = (np.asarray(case[k]) for k in ("line_from", "line_to", "line_b"))
    out = np.asarray(case["outaged"])
    assert len(set(out.tolist())) == len(out)
    assert np.all((frm != to) & (frm >= 0) & (to >= 0) & (frm < n) & (to < n))
    # a weighted Laplacian of a graph has one zero eigenvalue per component
    for drop in [None] + out.tolist():
        bb = b.copy()
        if drop is not None:
            bb[drop] = 0.0
        ev = np.linalg.eigvalsh(_laplacian(n, frm, to, bb))
        assert np.sum(ev < 1e-9 * ev.max()) == 1, drop


@pytest.mark.parametrize("case", [make_case("tiny"), make_case(scale_case(300, 24, 8, seed=5))],
                         ids=["tiny", "geometric_300"])
def test_limits_admit_the_capacity_proportional_dispatch(case):
    n, T = case["n_nodes"], case["T"]
    pmax = np.asarray(case["gen_pmax"])[:, 0]
    load = np.asarray(case["load_p"])
    inj = np.zeros((n, T))
    np.add.at(inj, case["gen_node"], (pmax / pmax.sum())[:, None] * load.sum(axis=0)[None, :])
    np.add.at(inj, case["load_node"], -load)
    u = np.asarray(case["line_u"])
    for drop in [None] + np.asarray(case["outaged"]).tolist():
        f = _dense_flows(case, inj, drop)
        assert np.all(np.abs(f) <= u[:, None] / 1.2 + 1e-9), drop
    assert np.all(u >= 0.5)


def test_device_draws_follow_the_recipe():
    c = make_case("2k")
    assert np.all((c["line_b"] >= 5) & (c["line_b"] <= 20))
    assert np.all((c["gen_a"] >= 0.01) & (c["gen_a"] <= 0.1))
    assert np.all((c["gen_b"] >= 10) & (c["gen_b"] <= 40))
    pmax = c["gen_pmax"]
    assert np.all(c["gen_pmin"] == 0) and np.all((pmax >= 1) & (pmax <= 3))
    assert np.all(pmax == pmax[:, :1])                         # constant over the horizon
    np.testing.assert_allclose(c["gen_ramp"], 0.2 * pmax[:, 0])
    assert np.all(c["load_voll"] == VOLL)                       # all load curtailable
    assert np.all(c["load_p"] > 0)
    # the daily profile: mean over loads follows 1 + 0.3 sin(2 pi t / 24 + phi)
    prof = c["load_p"].mean(axis=0) / c["load_p"].mean()
    assert prof.max() / prof.min() > 1.3
    assert np.all((c["stor_P"] >= 0.5) & (c["stor_P"] <= 2))
    assert np.all(c["stor_dur"] == 4) and np.all(c["stor_eff"] == 0.95)
    assert np.all((c["stor_cost"] >= 0) & (c["stor_cost"] <= 1))
    t = make_case("tiny")
    assert np.all(t["load_voll"] < 0) and np.all(t["gen_ramp"] < 0)   # fixed loads, no ramps
    assert len(t["stor_node"]) == 0


def test_hvdc_links_join_distinct_node_pairs():
    c = make_case(scale_case(50, 4, 2, seed=3, n_hvdc=6))
    pairs = {frozenset(p) for p in zip(c["hvdc_from"].tolist(), c["hvdc_to"].tolist())}
    assert len(pairs) == 6 and all(len(p) == 2 for p in pairs)
    assert np.all((c["hvdc_u"] >= 1) & (c["hvdc_u"] <= 3))
    # links are drawn last: the rest of the instance is the one without links
    base = make_case(scale_case(50, 4, 2, seed=3))
    for k in ("line_from", "line_u", "gen_pmax", "load_p", "outaged"):
        np.testing.assert_array_equal(c[k], base[k])
