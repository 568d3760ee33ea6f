"""The FP64 oracle sharded by contingency over single-threaded CPU processes,
compared on the fly with a state exported from the GPU path.

Test infrastructure: the parity tests at the benchmark's full sizes use it
to run the oracle for more iterations than one process finishes in
reasonable time.  Each rank holds a contiguous block of the contingencies
(``oracle.Shard``; the iteration couples contingencies only through the sums
over k of Section 3.2 step 2 and the residual norms of Section 3.3, which
the ranks all-reduce over gloo), runs the iterations, and compares its block
of every state array with the same block of the GPU state, which it reads
memory-mapped from ``.npy`` files.  Only squared norms travel between ranks,
so no process ever holds the whole oracle state.

Processes are started with ``spawn`` (the caller has already initialised
CUDA; a forked child of a CUDA process can hang).
"""
import json
import os
import socket

import numpy as np

STATE_KEYS = ("p_line", "th1", "th2", "v1", "v2", "p_dev", "u")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def save_state(state, out_dir):
    """Write the GPU state arrays (dict of host arrays) as .npy files."""
    for k in STATE_KEYS:
        np.save(os.path.join(out_dir, k + ".npy"), np.ascontiguousarray(state[k]))


def _rank_main(rank, world, port, case_spec, opts, n_iter, state_dir):
    import torch
    import torch.distributed as dist
    from gridgen import make_case, scale_case
    from oracle import Oracle, OracleOptions, Shard

    torch.set_num_threads(1)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        case = make_case(case_spec if isinstance(case_spec, str) else scale_case(**case_spec))
        K = len(case["outaged"])
        k_ids = np.array_split(np.arange(K + 1), world)[rank]

        def allreduce(x):
            t = torch.from_numpy(np.ascontiguousarray(x, np.float64)).clone()
            dist.all_reduce(t)
            return t.numpy()

        o = Oracle(case, OracleOptions(**opts), shard=Shard(k_ids, K, allreduce))
        o.iterate(n_iter, stop=False)
        L = o.net.L
        ref = dict(p_line=o.line_p(), th1=o.th[:, :L], th2=o.th[:, L:], v1=o.v[:, :L], v2=o.v[:, L:],
                   u=o.u)
        sums = np.zeros((len(STATE_KEYS), 2))
        for i, k in enumerate(STATE_KEYS):
            g = np.load(os.path.join(state_dir, k + ".npy"), mmap_mode="r")
            if k == "p_dev":
                if rank != 0:        # one schedule for every contingency: counted once
                    continue
                r, gk = o.dev_p(), np.asarray(g, np.float64)
            else:
                r, gk = ref[k], np.asarray(g[k_ids[0]:k_ids[-1] + 1], np.float64)
            assert gk.shape == r.shape, (k, gk.shape, r.shape)
            sums[i, 0] = np.sum((gk - r) ** 2)
            sums[i, 1] = np.sum(r * r)
        sums = allreduce(sums)
        if rank == 0:
            err = {k: float(np.sqrt(sums[i, 0]) / max(np.sqrt(sums[i, 1]), 1e-300))
                   for i, k in enumerate(STATE_KEYS)}
            scale = float(np.sqrt(sums[:, 1].max()))
            with open(os.path.join(state_dir, "oracle.json"), "w") as f:
                json.dump({"rel_err": err, "res": [float(x) for x in o.res], "rho": [o.rho_p, o.rho_th],
                           "rho_history": [list(h) for h in o.rho_history], "it": o.it,
                           "state_scale": scale}, f)
    finally:
        dist.destroy_process_group()


def compare_with_sharded_oracle(case_spec, opts, n_iter, gpu_state, state_dir, world=None):
    """Run the oracle for ``n_iter`` iterations from zero over ``world``
    processes (default: the host's cores, at most one per contingency) and
    return, for every state array, ``||X_gpu - X_oracle|| / ||X_oracle||``,
    with the oracle's residuals and penalty history.  ``case_spec`` is a
    named workload or ``scale_case`` keyword arguments (each rank builds the
    instance itself)."""
    import torch.multiprocessing as mp
    from gridgen import make_case, scale_case
    save_state(gpu_state, state_dir)
    if world is None:
        K = len(make_case(case_spec if isinstance(case_spec, str) else scale_case(**case_spec))["outaged"])
        world = max(1, min(os.cpu_count() or 1, K + 1, 16))
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        mp.start_processes(_rank_main, args=(world, _free_port(), case_spec, dict(opts), n_iter, state_dir),
                           nprocs=world, join=True, start_method="spawn")
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    with open(os.path.join(state_dir, "oracle.json")) as f:
        out = json.load(f)
    out["world"] = world
    return out
