"""Seeded synthetic instances with the shapes of the paper's workloads.

The paper's experiments run on PyPSA-USA Western Interconnect cases (Section 5
and Appendix E), which are not available here; these generators stand in for
them.  Each instance is a plain dict of NumPy arrays in the layout the
``opf_create`` C entry point takes:

* ``line_from``/``line_to`` (int32 node ids), ``line_b`` (susceptance),
  ``line_u`` (flow limit) -- the two-terminal AC lines of Section 2.1, which
  are the contingency device type;
* ``gen_*`` -- quadratic-cost generators ``a p^2 + b p`` with per-step box
  limits ``gen_pmin``/``gen_pmax`` (shape ``[n_gens, T]``) and an optional ramp
  limit ``gen_ramp`` (``< 0`` means none);
* ``load_*`` -- loads with a consumption profile ``load_p`` (``[n_loads, T]``,
  positive = consumed) and ``load_voll`` (``< 0``: fixed load; otherwise a
  curtailable load whose curtailment costs ``voll`` per unit);
* ``stor_*`` -- batteries with power ``P``, duration ``dur`` (in steps),
  charge efficiency ``eff`` and discharge cost ``cost`` (Section 2.1);
* ``outaged`` -- for contingency ``k = 1..K`` the index of the line that is
  out (Section 2.3, N-1 example).

The recipe (all draws from one ``numpy.random.default_rng(seed)`` stream):

* topology: ``tiny`` uses a random spanning tree plus random extra edges;
  the other sizes place buses uniformly in the unit square and take the
  Euclidean minimum spanning tree plus the shortest remaining Delaunay edges
  (grid-like locality, average degree ``2 L / N``);
* susceptance ``U[5, 20]``; flow limits ``max(U[0.5, 2], 1.2 * |f|)`` where
  ``f`` is the largest DC power flow of the line over every step and every
  contingency under a dispatch proportional to generator capacity.  That
  floor makes every instance feasible: the proportional dispatch is shared by
  all contingencies and respects every limit;
* generators: ``a ~ U[0.01, 0.1]``, ``b ~ U[10, 40]``, ``pmin = 0``,
  ``pmax ~ U[1, 3]``, ramp limit ``0.2 pmax`` per step when enabled;
* loads: base ``U[0.1, 0.5]`` times ``1 + 0.3 sin(2 pi t / 24 + phi)`` (phase
  ``phi ~ U[-pi/6, pi/6]`` per load) times ``lognormal(0, 0.1)`` per (load, t);
  fixed (``tiny``) or curtailable at ``VOLL = 500``;
* storage: ``P ~ U[0.5, 2]``, duration 4 steps, efficiency 0.95,
  discharge cost ``U[0, 1]``;
* contingencies: ``K`` distinct single-line outages drawn among lines whose
  removal keeps the grid connected (no islanding).

None of this is the method's arithmetic: the DC power flow only sets limits.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components, minimum_spanning_tree
from scipy.sparse.linalg import splu
from scipy.spatial import Delaunay

VOLL = 500.0

# Named workloads.  ``lines`` is the number of two-terminal lines.
CONFIGS = {
    # 30-bus, T=1, 5 outages, fixed loads, no storage, no ramps.
    "tiny": dict(n_nodes=30, n_lines=40, n_gens=6, n_loads=20, n_stor=0, T=1, K=5,
                 seed=0, topology="random_tree", fixed_frac=1.0, ramp=False),
    # 2,000 buses, ~3,200 lines, T=24, 20 outages.
    "2k": dict(n_nodes=2000, n_lines=3200, n_gens=500, n_loads=1500, n_stor=100, T=24,
               K=20, seed=1, topology="geometric", fixed_frac=0.0, ramp=True),
    # 10,000 buses, 15,000 lines, T=96 (four days, daily period 24), 50 outages.
    "10k": dict(n_nodes=10000, n_lines=15000, n_gens=2500, n_loads=7500, n_stor=500, T=96,
                K=50, seed=2, topology="geometric", fixed_frac=0.0, ramp=True),
    # the 10k network with 12 outages: per-contingency work of the 10k
    # instance at a quarter of its state (~1.1 GB, still far above L2), the
    # size on which kernel counters are captured
    "10k-K12": dict(n_nodes=10000, n_lines=15000, n_gens=2500, n_loads=7500, n_stor=500, T=96,
                    K=12, seed=2, topology="geometric", fixed_frac=0.0, ramp=True),
}


def scale_case(n_nodes, T, K, seed, *, lines_per_node=1.6, fixed_frac=0.0, ramp=True,
               stor_per_node=0.05, gens_per_node=0.25, loads_per_node=0.75,
               topology="geometric", n_hvdc=0):
    """Config dict for an arbitrary size with the 2k/10k device mix."""
    n_lines = max(n_nodes - 1, int(round(lines_per_node * n_nodes)))
    return dict(n_nodes=int(n_nodes), n_lines=int(n_lines),
                n_gens=max(1, int(round(gens_per_node * n_nodes))),
                n_loads=max(1, int(round(loads_per_node * n_nodes))),
                n_stor=int(round(stor_per_node * n_nodes)), T=int(T), K=int(K), seed=int(seed),
                topology=topology, fixed_frac=float(fixed_frac), ramp=bool(ramp), n_hvdc=int(n_hvdc))


def case_dims(case):
    """Sizes of an instance: N, L, gens, loads, storage, HVDC links, T, K,
    single-schedule terminals S (two per HVDC link) and terminals J."""
    L = len(case["line_from"])
    H = len(case.get("hvdc_from", ()))
    S = len(case["gen_node"]) + len(case["load_node"]) + len(case["stor_node"]) + 2 * H
    return dict(N=int(case["n_nodes"]), L=L, G=len(case["gen_node"]), D=len(case["load_node"]),
                B=len(case["stor_node"]), H=H, T=int(case["T"]), K=len(case["outaged"]),
                J=2 * L + S, S=S)


# ----------------------------------------------------------------------------
# topology
# ----------------------------------------------------------------------------

def _random_tree_topology(rng, n, n_lines):
    edges = set()
    frm, to = [], []
    for i in range(1, n):
        j = int(rng.integers(0, i))
        frm.append(j)
        to.append(i)
        edges.add((min(i, j), max(i, j)))
    max_edges = n * (n - 1) // 2
    if n_lines > max_edges:
        raise ValueError("too many lines for a simple graph")
    while len(frm) < n_lines:
        a, b = (int(x) for x in rng.integers(0, n, size=2))
        if a == b:
            continue
        e = (min(a, b), max(a, b))
        if e in edges:
            continue
        edges.add(e)
        frm.append(e[0])
        to.append(e[1])
    return np.asarray(frm, np.int64), np.asarray(to, np.int64), None


def _geometric_topology(rng, n, n_lines):
    xy = rng.random((n, 2))
    if n == 1:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), xy
    if n <= 3:
        pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    else:
        tri = Delaunay(xy)
        s = tri.simplices
        pe = np.concatenate([s[:, [0, 1]], s[:, [1, 2]], s[:, [0, 2]]], axis=0)
        pe.sort(axis=1)
        pe = np.unique(pe, axis=0)
        pairs = [tuple(e) for e in pe]
    pairs = np.asarray(pairs, np.int64)
    length = np.linalg.norm(xy[pairs[:, 0]] - xy[pairs[:, 1]], axis=1)
    W = coo_matrix((length + 1e-12, (pairs[:, 0], pairs[:, 1])), shape=(n, n)).tocsr()
    mst = minimum_spanning_tree(W).tocoo()
    tree = set()
    for a, b in zip(mst.row, mst.col):
        tree.add((min(a, b), max(a, b)))
    order = np.argsort(length, kind="stable")
    extra = [tuple(pairs[i]) for i in order if tuple(pairs[i]) not in tree]
    n_extra = n_lines - len(tree)
    if n_extra > len(extra):
        raise ValueError("not enough Delaunay edges for the requested line count")
    chosen = sorted(tree) + extra[:max(0, n_extra)]
    chosen = np.asarray(chosen, np.int64)
    # random orientation of each line
    flip = rng.random(len(chosen)) < 0.5
    frm = np.where(flip, chosen[:, 1], chosen[:, 0])
    to = np.where(flip, chosen[:, 0], chosen[:, 1])
    return frm, to, xy


def _connected_without(n, frm, to, drop):
    keep = np.ones(len(frm), bool)
    keep[drop] = False
    A = coo_matrix((np.ones(keep.sum()), (frm[keep], to[keep])), shape=(n, n))
    ncomp, _ = connected_components(A, directed=False)
    return ncomp == 1


def _dc_flows(n, frm, to, bsus, inj, drop=None):
    """Largest |DC flow| per line over the columns of ``inj`` ([n, T])."""
    keep = np.ones(len(frm), bool)
    if drop is not None:
        keep[drop] = False
    f, t, b = frm[keep], to[keep], bsus[keep]
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([b, b, -b, -b])
    Bm = coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsc()
    out = np.zeros(len(frm))
    if n == 1:
        return out
    red = Bm[1:, 1:].tocsc()
    lu = splu(red)
    th = np.zeros((n, inj.shape[1]))
    th[1:] = lu.solve(np.ascontiguousarray(inj[1:]))
    flow = b[:, None] * (th[f] - th[t])
    out[keep] = np.abs(flow).max(axis=1)
    return out


# ----------------------------------------------------------------------------
# instance
# ----------------------------------------------------------------------------

def make_case(cfg="tiny", seed=None, **overrides):
    """Draw one instance.  ``cfg`` is a name from ``CONFIGS`` or a config dict."""
    if isinstance(cfg, str):
        name = cfg
        cfg = dict(CONFIGS[cfg])
    else:
        cfg = dict(cfg)
        name = cfg.pop("name", "custom")
    cfg.update(overrides)
    if seed is not None:
        cfg["seed"] = seed
    rng = np.random.default_rng(cfg["seed"])
    n, L = cfg["n_nodes"], cfg["n_lines"]
    G, D, B, T, K = cfg["n_gens"], cfg["n_loads"], cfg["n_stor"], cfg["T"], cfg["K"]
    if L < n - 1:
        raise ValueError("a connected grid needs at least n_nodes - 1 lines")

    if cfg.get("topology", "geometric") == "random_tree":
        frm, to, xy = _random_tree_topology(rng, n, L)
    else:
        frm, to, xy = _geometric_topology(rng, n, L)

    bsus = rng.uniform(5.0, 20.0, L)
    u_draw = rng.uniform(0.5, 2.0, L)

    gen_node = rng.integers(0, n, G)
    gen_a = rng.uniform(0.01, 0.1, G)
    gen_b = rng.uniform(10.0, 40.0, G)
    pmax = rng.uniform(1.0, 3.0, G)
    gen_pmin = np.zeros((G, T))
    gen_pmax = np.repeat(pmax[:, None], T, axis=1)
    gen_ramp = 0.2 * pmax if (cfg.get("ramp", False) and T > 1) else -np.ones(G)

    load_node = rng.integers(0, n, D)
    base = rng.uniform(0.1, 0.5, D)
    phase = rng.uniform(-math.pi / 6, math.pi / 6, D)
    t = np.arange(T)
    shape = 1.0 + 0.3 * np.sin(2.0 * math.pi * t[None, :] / 24.0 + phase[:, None])
    noise = rng.lognormal(0.0, 0.1, (D, T))
    load_p = base[:, None] * shape * noise
    n_fixed = int(round(cfg.get("fixed_frac", 0.0) * D))
    load_voll = np.full(D, VOLL)
    if n_fixed:
        load_voll[rng.permutation(D)[:n_fixed]] = -1.0

    stor_node = rng.integers(0, n, B)
    stor_P = rng.uniform(0.5, 2.0, B)
    stor_dur = np.full(B, 4.0)
    stor_eff = np.full(B, 0.95)
    stor_cost = rng.uniform(0.0, 1.0, B)

    # K distinct non-islanding single-line outages
    outaged = []
    if K:
        for l in rng.permutation(L):
            if _connected_without(n, frm, to, int(l)):
                outaged.append(int(l))
                if len(outaged) == K:
                    break
        if len(outaged) < K:
            raise ValueError("not enough non-bridge lines for the requested outages")

    # limit floor from a capacity-proportional dispatch (keeps every case feasible)
    demand = load_p.sum(axis=0)
    share = pmax / pmax.sum() if G else np.zeros(0)
    inj = np.zeros((n, T))
    np.add.at(inj, gen_node, share[:, None] * demand[None, :])
    np.add.at(inj, load_node, -load_p)
    fmax = _dc_flows(n, frm, to, bsus, inj) if L else np.zeros(0)
    for l in outaged:
        fmax = np.maximum(fmax, _dc_flows(n, frm, to, bsus, inj, drop=l))
    line_u = np.maximum(u_draw, 1.2 * fmax)

    # HVDC links (Section 2.1, other devices): distinct node pairs (no two
    # links join the same two nodes), limit U[1, 3]; drawn last so that cases
    # without them are unchanged
    H = int(cfg.get("n_hvdc", 0))
    pairs = []
    while len(pairs) < H:
        a, c = (int(v) for v in rng.choice(n, 2, replace=False))
        if (a, c) not in pairs and (c, a) not in pairs:
            pairs.append((a, c))
    hvdc_from = np.array([a for a, _ in pairs], np.int64)
    hvdc_to = np.array([c for _, c in pairs], np.int64)
    hvdc_u = rng.uniform(1.0, 3.0, H)

    return dict(
        name=name, seed=int(cfg["seed"]), T=int(T), n_nodes=int(n),
        line_from=frm.astype(np.int32), line_to=to.astype(np.int32),
        line_b=bsus, line_u=line_u,
        gen_node=gen_node.astype(np.int32), gen_a=gen_a, gen_b=gen_b,
        gen_pmin=gen_pmin, gen_pmax=gen_pmax, gen_ramp=gen_ramp,
        load_node=load_node.astype(np.int32), load_p=load_p, load_voll=load_voll,
        stor_node=stor_node.astype(np.int32), stor_P=stor_P, stor_dur=stor_dur,
        stor_eff=stor_eff, stor_cost=stor_cost,
        outaged=np.asarray(outaged, np.int32),
        hvdc_from=hvdc_from.astype(np.int32), hvdc_to=hvdc_to.astype(np.int32), hvdc_u=hvdc_u,
    )
