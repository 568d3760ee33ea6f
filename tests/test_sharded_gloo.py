"""Contingency sharding over several processes (gloo, CPU).

The iteration couples contingencies only through the sums over k that feed
the non-contingency proxes (Section 3.2) and through the residual norms
(Section 3.3).  Ranks each hold a contiguous block of the contingencies
(uneven blocks when K + 1 does not divide evenly), all-reduce
exactly those quantities, and must reproduce the single-process iteration:
the same states (to FP64 rounding of the split sums), residuals and
penalty decisions.  This is the exchange a contingency-sharded multi-GPU
run performs once per iteration.
"""
import os
import socket

import numpy as np
import pytest

from gridgen import make_case, scale_case


def _case(hvdc=False):
    return make_case(scale_case(60, 6, 5, seed=31, n_hvdc=3 if hvdc else 0))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, n_iter, alpha=1.0, hvdc=False):
    import torch
    import torch.distributed as dist
    from oracle import Oracle, OracleOptions, Shard

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        case = _case(hvdc)
        K = len(case["outaged"])
        k_ids = np.array_split(np.arange(K + 1), world)[rank]

        def allreduce(x):
            t = torch.from_numpy(np.ascontiguousarray(x, np.float64)).clone()
            dist.all_reduce(t)
            return t.numpy()

        o = Oracle(case, OracleOptions(adapt_every=10, eps=0.0, alpha=alpha), shard=Shard(k_ids, K, allreduce))
        res = []
        for _ in range(n_iter):
            o.step()
            res.append(o.res.copy())
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), k_ids=k_ids, p=o.p, th=o.th, u=o.u, v=o.v,
                 res=np.array(res), rho=np.array([o.rho_p, o.rho_th]),
                 hist=np.array(o.rho_history, float), prices=o.prices())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world, alpha, hvdc", [(2, 1.0, False), (2, 1.5, True), (4, 1.0, True)])
def test_contingency_shards_reproduce_the_iteration(tmp_path, world, alpha, hvdc):
    """Plain message passing, and the over-relaxed iteration (Section 3.6) on
    a grid with HVDC links (two-terminal devices shared by all contingencies);
    four ranks split the six contingency rows 2, 2, 1, 1."""
    import torch.multiprocessing as mp
    from oracle import Oracle, OracleOptions

    n_iter = 30
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path), n_iter, alpha, hvdc), nprocs=world,
                       join=True, start_method="spawn")
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]

    ref = Oracle(_case(hvdc), OracleOptions(adapt_every=10, eps=0.0, alpha=alpha))
    res = []
    for _ in range(n_iter):
        ref.step()
        res.append(ref.res.copy())
    res = np.array(res)

    for name in ("p", "th", "u", "v"):
        full = getattr(ref, name)
        got = np.concatenate([q[name] for q in parts], axis=0)
        assert got.shape == full.shape
        np.testing.assert_allclose(got, full, rtol=1e-10, atol=1e-12 * np.abs(full).max(), err_msg=name)
    for q in parts:
        np.testing.assert_allclose(q["res"], res, rtol=1e-10)
        assert q["rho"].tolist() == [ref.rho_p, ref.rho_th]
        assert q["hist"].tolist() == [list(h) for h in ref.rho_history]
        np.testing.assert_allclose(q["prices"], ref.prices(), rtol=1e-10, atol=1e-12)
    assert np.concatenate([q["k_ids"] for q in parts]).tolist() == list(range(ref.net.Kp))
    assert [len(q["k_ids"]) for q in parts] == [len(b) for b in np.array_split(np.arange(ref.net.Kp), world)]


def test_sharded_comparison_helper_finds_agreement_and_a_planted_error(tmp_path):
    """The helper the full-size GPU parity tests use: a state taken from the
    unsharded oracle compares at FP64 rounding, and the same state with one
    entry of one contingency changed is reported for that array only."""
    from helpers import oracle_arrays
    from oracle import Oracle, OracleOptions
    from sharded_oracle import compare_with_sharded_oracle
    spec = dict(n_nodes=40, T=4, K=5, seed=33)
    opts = dict(adapt_every=10, eps=0.0)
    ref = Oracle(make_case(scale_case(**spec)), OracleOptions(**opts))
    ref.iterate(25, stop=False)
    st = {k: np.array(v) for k, v in oracle_arrays(ref).items()}
    (tmp_path / "a").mkdir()
    out = compare_with_sharded_oracle(spec, opts, 25, st, str(tmp_path / "a"), world=3)
    assert out["world"] == 3 and out["it"] == 25
    assert max(out["rel_err"].values()) < 1e-12
    np.testing.assert_allclose(out["res"], ref.res, rtol=1e-10)
    assert out["rho"] == [ref.rho_p, ref.rho_th]
    st["v2"][4, 7, 2] += 0.5 * np.abs(st["v2"]).max()
    (tmp_path / "b").mkdir()
    out = compare_with_sharded_oracle(spec, opts, 25, st, str(tmp_path / "b"), world=2)
    assert out["rel_err"]["v2"] > 1e-3
    assert max(v for k, v in out["rel_err"].items() if k != "v2") < 1e-12
