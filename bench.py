"""Benchmark: proximal message passing iterations/s on the 10k-bus workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one iteration of the whole hot path (every line prox in every
contingency, every device prox including the inner ADMM of ramp-limited
generators and batteries, node averages, price updates, FP64 residuals and
the adaptive penalty) over the 10,000-bus, T = 96, K = 50 synthetic instance.
``value`` is iterations/s with the state resident in HBM; under torchrun
each rank solves its own instance (independent problems, weak scaling, no
data-path collective) and ``value`` sums all ranks.  ``e2e`` is the same
metric through the C ABI with host buffers: network upload, the K
iterations and the solution download are inside the timed region.

``time_to_tolerance`` (skip with ``--no-ttt``): wall time and iterations to
the eps = 1e-4 test of Eq. (converge) with the adaptive penalty, through the C
ABI: the instance cold, the instance with every load scaled by
lognormal(0, 0.05) cold, and that perturbed instance warm-started from the
first solution (Section 3.4) kept on the device, and again imported from host
memory inside the timed region; and the instance cold with over-relaxation
alpha = 1.5 (Section 3.6; ``--ttt-alpha``).

``--adjoint K`` (default 200, 0 to skip): wall time of the cost gradient
after K unrolled iterations (include/opf_diff.h) on the 2k instance,
checkpoints every 20 iterations and every state kept.

``--impl reference`` times the FP64 oracle on the host cores instead; each
step is one oracle iteration on a bounded sample of the instance (the 10k
network with fewer contingencies and time steps), converted to full-workload
iterations/s by the paper's variable count 4 J T (K+1) per iteration.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADMM iterations/s"
UNIT = "iter/s"
def workload_name(config, d):
    """Name of the timed workload: the network size, horizon and contingencies."""
    return f"dcopf-{config}-bus-T{d['T']}-K{d['K']}"
KERNEL_SRC = [os.path.join(ROOT, "paper_2410_17203_gb300", "csrc", f)
              for f in ("opf_kernels.cu", "opf_internal.h")]
PROFILE = os.path.join(ROOT, "profiles", "iteration_10k.txt")
FALLBACK_HBM_GBS = 6800.0


def byte_model(d):
    """Algorithmic bytes of one iteration: every FP32 element of the method's
    state (Section 4.4) read once and written once -- lines p, theta1, theta2,
    v1, v2; nodes u, pbar, theta_bar (each [K+1][.][T]); device power [S][T].
    The library stores theta1, theta2 as their mean plus p (theta1 - theta2 =
    p / b after every line prox), so it moves less than this per iteration;
    the measured DRAM traffic is reported beside it."""
    Kp, T = d["K"] + 1, d["T"]
    return 8 * Kp * T * (5 * d["L"] + 3 * d["N"]) + 8 * d["S"] * T


def variables_per_iter(d):
    """The paper's problem-size convention 4 J T (K+1) (p, theta, u, v)."""
    return 4 * d["J"] * d["T"] * (d["K"] + 1)


def peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SRC:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per iteration from the committed ncu summary, if it was taken
    on the current kernel source."""
    try:
        kv = {}
        for line in open(PROFILE):
            if ":" in line:
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256") != kernel_hash():
            return None
        return float(kv["dram_bytes_per_iteration"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        load = [s for s in sm if mx and s > 0.3 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# the oracle on the host (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def sample_case(case, k_s, T_s):
    """The instance with its first k_s contingencies and first T_s steps."""
    import numpy as np
    c = dict(case)
    c["outaged"] = np.asarray(case["outaged"][:k_s], np.int32)
    c["T"] = T_s
    for k in ("gen_pmin", "gen_pmax", "load_p"):
        c[k] = np.ascontiguousarray(case[k][:, :T_s])
    if T_s <= 1:
        c["gen_ramp"] = -np.ones(len(case["gen_node"]))
    return c


def oracle_child(cfg, k_s, T_s, steps, warmup):
    """Runs in a child process with single-threaded BLAS: times the oracle."""
    from gridgen import case_dims, make_case
    from oracle import Oracle, OracleOptions
    c = sample_case(make_case(cfg), k_s, T_s)
    o = Oracle(c, OracleOptions(adapt_every=10, eps=0.0))
    for _ in range(warmup):
        o.step()
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step()
    dt = time.perf_counter() - t0
    d = case_dims(c)
    return {"seconds": dt, "steps": steps, "vars_per_iter": variables_per_iter(d),
            "K_sample": k_s, "T_sample": T_s}


def _oracle_rank(rank, world, port, cfg, k_s, T_s, steps, warmup, out):
    """One rank of the contingency-sharded oracle (gloo all-reduce of the
    sums over k and of the residual parts, single-threaded BLAS)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from gridgen import make_case
    from oracle import Oracle, OracleOptions, Shard
    torch.set_num_threads(1)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        c = sample_case(make_case(cfg), k_s, T_s)
        K = len(c["outaged"])
        k_ids = np.array_split(np.arange(K + 1), world)[rank]

        def allreduce(x):
            t = torch.from_numpy(np.ascontiguousarray(x, np.float64)).clone()
            dist.all_reduce(t)
            return t.numpy()

        o = Oracle(c, OracleOptions(adapt_every=10, eps=0.0), shard=Shard(k_ids, K, allreduce))
        for _ in range(warmup):
            o.step()
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            o.step()
        dist.barrier()
        dt = time.perf_counter() - t0
        if rank == 0:
            with open(out, "w") as f:
                json.dump({"seconds": dt}, f)
    finally:
        dist.destroy_process_group()


def oracle_child_sharded(cfg, k_s, T_s, steps, warmup, world):
    """Runs in a child process: the oracle over `world` single-threaded
    processes, each holding a share of the contingencies."""
    import socket
    import tempfile
    import torch.multiprocessing as mp
    from gridgen import case_dims, make_case
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    with tempfile.TemporaryDirectory() as td:
        out = os.path.join(td, "t.json")
        mp.start_processes(_oracle_rank, args=(world, port, cfg, k_s, T_s, steps, warmup, out), nprocs=world,
                           join=True, start_method="spawn")
        with open(out) as f:
            dt = json.load(f)["seconds"]
    d = case_dims(sample_case(make_case(cfg), k_s, T_s))
    return {"seconds": dt, "steps": steps, "vars_per_iter": variables_per_iter(d), "K_sample": k_s,
            "T_sample": T_s, "processes": world}


def run_oracle(cfg, k_s, T_s, steps, warmup, world=1):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    kw = dict(cfg=cfg, k_s=k_s, T_s=T_s, steps=steps, warmup=warmup)
    if world > 1:
        kw["world"] = world
    cmd = [sys.executable, os.path.abspath(__file__), "--_oracle-child", json.dumps(kw)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle child failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def host_cpu():
    """The host CPU's model as the OS reports it (x86: model name; Arm: the
    implementer / part codes and the lscpu model name when present)."""
    import platform
    info = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    info.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if "model name" in info:
        return info["model name"]
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    parts = [f"{k} {info[k]}" for k in ("CPU implementer", "CPU part") if k in info]
    return ", ".join(parts) or platform.machine()


def oracle_value(res, full_vars):
    """Full-workload iterations/s from the sample's variable-update rate."""
    upd = res["vars_per_iter"] * res["steps"] / res["seconds"]
    return upd / full_vars


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reference_arm(args):
    from gridgen import CONFIGS, case_dims, make_case
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    full = make_case(args.config)
    d = case_dims(full)
    # per-step budget: the whole run in about two minutes
    per_step = 120.0 / max(1, args.steps + args.warmup)
    # oracle cost is about 0.4 s per (contingency, 96 steps) at 10k on one core
    unit = 0.4 * d["T"] / 96.0 * (d["N"] / 10000.0)
    k_s = max(0, min(d["K"], int(per_step / unit) - 1))
    T_s = d["T"] if k_s > 0 else max(1, min(d["T"], int(d["T"] * per_step / unit)))
    res = run_oracle(args.config, k_s, T_s, args.steps, args.warmup)
    v = oracle_value(res, variables_per_iter(d))
    sample = (f"{args.config} network, contingencies 0..{k_s}, steps 0..{T_s - 1}; "
              f"value scaled by 4JT(K+1) variables per iteration")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * res["seconds"] / res["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(args.config, d), "N": d["N"], "L": d["L"], "T": d["T"], "K": d["K"],
                       "S": d["S"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu": host_cpu(), "host_cores": os.cpu_count()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def solve_to_tolerance(case, stream, args, opts=None, state=None, state_on_device=False):
    """Iterate to eps = 1e-4 through the C ABI; wall time includes the state
    import of a warm start (host arrays, or CUDA tensors with
    state_on_device).  Returns (info, seconds, handle)."""
    import torch
    from paper_2410_17203_gb300 import opf_create, opf_get_info, opf_iterate, opf_set_state
    o = dict(adapt_every=10, eps=1e-4)
    o.update(opts or {})
    h = opf_create(case, o, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if state is not None:
        opf_set_state(h, state, on_device=state_on_device)
    done = 0
    while done < args.ttt_max:
        opf_iterate(h, args.ttt_chunk)
        done += args.ttt_chunk
        if opf_get_info(h)["converged"]:
            break
    dt = time.perf_counter() - t0
    return opf_get_info(h), dt, h


def time_to_tolerance(case, stream, args):
    import numpy as np
    from paper_2410_17203_gb300 import opf_destroy, opf_get_state, opf_residuals

    def entry(info, dt, h):
        return {"converged": bool(info["converged"]), "iterations": int(info["iterations"]),
                "seconds": dt, "residuals": [float(x) for x in opf_residuals(h)[:2]],
                "tolerance": info["tolerance"]}

    import torch
    from paper_2410_17203_gb300 import state_shapes

    info, dt, h = solve_to_tolerance(case, stream, args)
    out = {"eps": 1e-4, "cold": entry(info, dt, h)}
    state = opf_get_state(h)
    # the same solution kept on the device (in HBM, as a solver that keeps its
    # previous solution would)
    dstate = {k: torch.zeros(sh, dtype=torch.float32, device="cuda") for k, sh in state_shapes(info).items()}
    opf_get_state(h, on_device=True, out=dstate)
    torch.cuda.synchronize()
    rho = (info["rho_p"], info["rho_theta"])
    opf_destroy(h)
    # the same network with every load scaled by lognormal(0, 0.05) per step
    rng = np.random.default_rng(12345)
    pert = dict(case)
    pert["load_p"] = case["load_p"] * rng.lognormal(0.0, 0.05, size=case["load_p"].shape)
    info, dt, h = solve_to_tolerance(pert, stream, args)
    out["perturbed_cold"] = entry(info, dt, h)
    opf_destroy(h)
    info, dt, h = solve_to_tolerance(pert, stream, args, opts=dict(rho_p=rho[0], rho_theta=rho[1]),
                                     state=dstate, state_on_device=True)
    out["perturbed_warm"] = entry(info, dt, h)
    out["perturbed_warm"]["state"] = "the previous solution on the device"
    opf_destroy(h)
    info, dt, h = solve_to_tolerance(pert, stream, args, opts=dict(rho_p=rho[0], rho_theta=rho[1]),
                                     state=state)
    out["perturbed_warm_host_state"] = entry(info, dt, h)
    out["perturbed_warm_host_state"]["state"] = "the previous solution in host memory (imported in the timed region)"
    opf_destroy(h)
    out["perturbation"] = "load_p x lognormal(0, 0.05) per (load, step), seed 12345"
    if args.ttt_alpha != 1.0:
        # the instance cold with over-relaxation (Section 3.6)
        info, dt, h = solve_to_tolerance(case, stream, args, opts=dict(alpha=args.ttt_alpha))
        out[f"cold_alpha_{args.ttt_alpha:g}"] = entry(info, dt, h)
        opf_destroy(h)
    return out


def batch_instances(n, seed=3):
    """The batched workload: n independent instances, buses log-uniform in
    [100, 5000], T uniform in {1, 24, 48}, 0..20 outages, the device mix of the
    other workloads (generators N/4, loads 3N/4, batteries N/20, lines 1.5 N)."""
    import numpy as np
    from gridgen import make_case, scale_case
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nb = int(round(float(np.exp(rng.uniform(np.log(100), np.log(5000))))))
        T = int(rng.choice([1, 24, 48]))
        K = int(rng.integers(0, 21))
        out.append(make_case(scale_case(nb, T, K, seed=1000 + i, lines_per_node=1.5)))
    return out


def batched_vs_plain(stream, args):
    """Solve every instance to eps = 1e-4: one after another through
    opf_iterate (plain), and all at once through one batch graph.  With the
    stall rule (--stall-window) an instance on which the adaptive penalty
    cycles has its penalties fixed and goes on; one that stops falling at
    fixed penalties stops with OPF_ESTALLED."""
    import torch
    from paper_2410_17203_gb300 import (BATCH_LAYOUTS, opf_batch_autotune, opf_batch_compact, opf_batch_create,
                                        opf_batch_destroy, opf_batch_iterate, opf_batch_stopped, opf_create,
                                        opf_destroy, opf_get_info, opf_iterate, opf_reset)
    cases = batch_instances(args.batched)
    opts = dict(adapt_every=10, eps=1e-4, stall_window=args.stall_window)
    chunk = args.ttt_chunk
    plain = [opf_create(c, opts, stream=stream.cuda_stream) for c in cases]
    batch = [opf_create(c, opts, stream=stream.cuda_stream) for c in cases]
    b = opf_batch_create(batch)
    # build every graph once, then start from zero again
    for h in plain:
        opf_iterate(h, 17)
    opf_batch_iterate(b, 17)
    torch.cuda.synchronize()
    for h in plain + batch:
        opf_reset(h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its_plain = []
    for h in plain:
        done = 0
        while done < args.ttt_max:
            opf_iterate(h, chunk)
            done += chunk
            i = opf_get_info(h)
            if i["converged"] or i["stalled"]:
                break
        its_plain.append(int(opf_get_info(h)["iterations"]))
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    choice, layout_ms = opf_batch_autotune(b, steps=20)    # from the zero state, which it restores
    t_tune = time.perf_counter() - t0
    done, sched, n_compact = 0, len(batch), 0
    while done < args.ttt_max:
        opf_batch_iterate(b, chunk)
        done += chunk
        stopped = sum(opf_batch_stopped(b))
        if stopped == len(batch):
            break
        if len(batch) - stopped <= 0.75 * sched:        # schedule the running instances only
            sched = opf_batch_compact(b)
            n_compact += 1
    t_batch = time.perf_counter() - t0
    infos = [opf_get_info(h) for h in batch]
    its_batch = [int(i["iterations"]) for i in infos]
    n_conv, n_stall, n_err = opf_batch_stopped(b)
    n_frozen_conv = sum(1 for i in infos if i["converged"] and i["frozen_at"] > 0)
    opf_batch_destroy(b)
    for h in plain + batch:
        opf_destroy(h)
    return {"instances": len(cases), "eps": 1e-4, "stall_window": args.stall_window,
            "plain_seconds": t_plain, "batched_seconds": t_batch, "speedup": t_plain / t_batch,
            "converged_batched": n_conv, "stalled_batched": n_stall, "error_batched": n_err,
            "at_cap_batched": len(batch) - n_conv - n_stall - n_err,
            "converged_after_fixing_penalties": n_frozen_conv,
            "iterations_total": int(sum(its_plain)),
            "iterations_equal": its_plain == its_batch,
            "compactions": n_compact,
            "autotune": {"seconds": t_tune, "chosen": BATCH_LAYOUTS[choice],
                         "ms_per_batch_iteration": dict(zip(BATCH_LAYOUTS, layout_ms))},
            "workload": "buses log-uniform [100, 5000], T in {1, 24, 48}, K in 0..20, seed 3"}


def batch_solve(handles, args):
    """Iterate a batch of contexts until every instance has stopped
    (converged, stalled) or the iteration cap; returns (iterations per
    instance, converged flags, seconds including the autotuner)."""
    from paper_2410_17203_gb300 import (opf_batch_autotune, opf_batch_compact, opf_batch_create,
                                        opf_batch_destroy, opf_batch_iterate, opf_batch_stopped, opf_get_info)
    b = opf_batch_create(handles)
    t0 = time.perf_counter()
    opf_batch_autotune(b, steps=20)
    done, sched = 0, len(handles)
    while done < args.ttt_max:
        opf_batch_iterate(b, args.ttt_chunk)
        done += args.ttt_chunk
        stopped = sum(opf_batch_stopped(b))
        if stopped == len(handles):
            break
        if len(handles) - stopped <= 0.75 * sched:      # schedule the running instances only
            sched = opf_batch_compact(b)
    dt = time.perf_counter() - t0
    its = [int(opf_get_info(h)["iterations"]) for h in handles]
    conv = [bool(opf_get_info(h)["converged"]) for h in handles]
    opf_batch_destroy(b)
    return its, conv, dt


def learned_warm_start(stream, args):
    """The learned warm start against a cold start and against the paper's own
    warm start (Section 3.4: the whole solution of the unperturbed network,
    with its final penalties), on the same held-out load-perturbed copies of
    the 2k network, all solved to eps = 1e-4.  The network is trained on the
    other copies' solutions (reached from the Section 3.4 start), with the
    library's kernels; its output becomes the starting state on the device
    (opf_set_state_from_nodes)."""
    import numpy as np
    import torch
    from gridgen import make_case
    from paper_2410_17203_gb300 import (WarmStartNet, opf_create, opf_destroy, opf_get_info, opf_get_state,
                                        opf_set_state, opf_set_state_from_nodes, opf_solution)
    from paper_2410_17203_gb300 import warmstart as ws

    base = make_case("2k")
    n_all = args.learned
    n_test = min(64, max(1, n_all // 4))
    rng = np.random.default_rng(4)
    cases = []
    for i in range(n_all):
        c = dict(base)
        c["load_p"] = base["load_p"] * rng.lognormal(0.0, 0.15, size=base["load_p"].shape)
        cases.append(c)
    opts = dict(adapt_every=10, eps=1e-4)
    N, T = base["n_nodes"], base["T"]
    Kp = len(base["outaged"]) + 1
    # the unperturbed network's solution: the Section 3.4 starting point
    h0 = opf_create(base, opts, stream=stream.cuda_stream)
    its0, _, _ = batch_solve([h0], args)
    i0 = opf_get_info(h0)
    S0 = opf_get_state(h0)
    opf_destroy(h0)
    wopts = dict(opts, rho_p=i0["rho_p"], rho_theta=i0["rho_theta"])
    # 1. every copy from the Section 3.4 start (batches of at most 128
    #    contexts): training targets, and the baseline of the held-out copies
    its_nom, conv_nom, t_nom, Y = [], [], [], []
    for c0 in range(0, n_all, 128):
        hs = [opf_create(c, wopts, stream=stream.cuda_stream) for c in cases[c0:c0 + 128]]
        t0 = time.perf_counter()
        for h in hs:
            opf_set_state(h, S0)
        its, conv, dt = batch_solve(hs, args)
        its_nom += its
        conv_nom += conv
        t_nom.append(time.perf_counter() - t0)
        for h in hs:
            price = np.zeros((N, T), np.float32)
            theta = np.zeros((Kp, N, T), np.float32)
            opf_solution(h, False, False, theta_node=theta, price=price)
            Y.append(ws.targets(price, theta[0]))
            opf_destroy(h)
    X = [ws.node_features(c) for c in cases]
    train_idx = [i for i in range(n_all - n_test) if conv_nom[i]]
    test_idx = list(range(n_all - n_test, n_all))
    norm = ws.Normalizer(np.concatenate([X[i] for i in train_idx]))
    ystd = np.concatenate([Y[i] for i in train_idx]).std(axis=0)
    scale = tuple(float(1.0 / max(v * v, 1e-12)) for v in ystd)
    dev = torch.device("cuda", torch.cuda.current_device())
    xd = [torch.from_numpy(norm(x)).to(dev) for x in X]
    yd = [torch.from_numpy(y.astype(np.float32)).to(dev) for y in Y]
    # 2. train on the GPU with the library's kernels
    net = WarmStartNet(N, base["line_from"], base["line_to"], base["line_b"], T, ws.N_FEATURES, seed=1,
                       stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = ws.train(net, [xd[i] for i in train_idx], [yd[i] for i in train_idx], args.learned_epochs,
                    args.learned_lr, scale=scale)
    t_train = time.perf_counter() - t0
    test_loss = float(np.mean([net.gradient(xd[i], yd[i], scale)[0] for i in test_idx]))
    # 3. the held-out copies: cold, and from the network's start (built on the device)
    hc = [opf_create(cases[i], opts, stream=stream.cuda_stream) for i in test_idx]
    its_cold, conv_cold, t_cold = batch_solve(hc, args)
    for h in hc:
        opf_destroy(h)
    hw = [opf_create(cases[i], opts, stream=stream.cuda_stream) for i in test_idx]
    y = torch.zeros((N * T, 2), dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    for h, i in zip(hw, test_idx):
        net.forward(xd[i], y)
        opf_set_state_from_nodes(h, y, ws.PRICE_SCALE, on_device=True)
    t_start = time.perf_counter() - t0
    its_learned, conv_learned, t_learned = batch_solve(hw, args)
    for h in hw:
        opf_destroy(h)
    net.close()
    nom = [its_nom[i] for i in test_idx]

    def summary(its, conv, seconds):
        return {"mean": float(np.mean(its)), "median": float(np.median(its)), "converged": int(sum(conv)),
                "seconds_batched": seconds}
    return {"network": "2k buses, T=24, K=20; loads x lognormal(0, 0.15) per (load, step), seed 4; "
                       f"the last {n_test} copies held out",
            "instances": n_all, "train": len(train_idx), "test": len(test_idx),
            "epochs": args.learned_epochs, "lr": args.learned_lr,
            "train_loss_first_last": [hist[0], hist[-1]], "test_loss": test_loss, "train_seconds": t_train,
            "test_iterations_cold": summary(its_cold, conv_cold, t_cold),
            "test_iterations_learned": summary(its_learned, conv_learned, t_learned + t_start),
            "test_iterations_section_3_4_start": summary(nom, [conv_nom[i] for i in test_idx], None),
            "section_3_4_start": "the unperturbed network's solution and final penalties "
                                 f"({int(its0[0])} iterations cold)"}


def adjoint_leg(stream, args):
    """Cost and gradient after K unrolled iterations (include/opf_diff.h) on
    the 2k instance (ramp-limited generators and batteries through the inner
    ADMM): wall time of one forward + reverse pass against the forward alone
    (medians of five calls each, alternating)."""
    import numpy as np
    import torch
    from gridgen import make_case
    from paper_2410_17203_gb300 import UnrolledCost

    case = make_case("2k")
    K = args.adjoint

    def timed(ck):
        d = UnrolledCost(case, rho_p=1.0, rho_theta=1.0, checkpoint_every=ck, stream=stream.cuda_stream)
        try:
            d.cost_grad(K)                               # warm-up (allocations, module load)
            t_fg, t_f = [], []
            for _ in range(5):
                t0 = time.perf_counter()
                f, g = d.cost_grad(K)
                t_fg.append(time.perf_counter() - t0)
                t0 = time.perf_counter()
                d.cost_grad(K, grads=False)
                t_f.append(time.perf_counter() - t0)
        finally:
            d.close()
        torch.cuda.synchronize()
        return f, g, float(np.median(t_fg)), float(np.median(t_f))

    f, g, t_fg, t_f = timed(20)
    f1, g1, t_fg1, t_f1 = timed(1)                       # every state kept: no recomputation
    return {"network": "2k instance: 2000 buses, T=24, K=20, 500 ramp-limited generators, 1500 curtailable "
                       "loads, 100 batteries, seed 1; gradients w.r.t. loads, capacities and line limits",
            "iterations": K, "checkpoint_every": 20, "seconds_cost_and_gradient": t_fg,
            "seconds_cost_only": t_f, "cost": f,
            "grad_norms": {k: float(np.linalg.norm(v)) for k, v in g.items()},
            "every_state_kept": {"checkpoint_every": 1, "seconds_cost_and_gradient": t_fg1,
                                 "seconds_cost_only": t_f1,
                                 "same_gradients": bool(f1 == f and all(np.array_equal(g1[k], g[k]) for k in g))}}


class PlainRunner:
    """One context over the whole instance, iterated by opf_iterate."""

    def __init__(self, case, opts, stream):
        from paper_2410_17203_gb300 import opf_create
        self.h = opf_create(case, opts, stream=stream.cuda_stream)

    def run(self, n):
        from paper_2410_17203_gb300 import opf_iterate
        opf_iterate(self.h, n)

    def close(self):
        from paper_2410_17203_gb300 import opf_destroy
        opf_destroy(self.h)


class SliceRunner:
    """This rank's block of the contingencies (include/opf.h, contingency
    slices): per iteration the local half, an all-reduce of the exchange
    buffer on the context's stream, and the decisions."""

    def __init__(self, case, opts, stream, dist, ws, rank):
        import numpy as np
        import torch
        from paper_2410_17203_gb300 import opf_create_slice, opf_slice_exchange, opf_slice_prime
        blocks = np.array_split(np.arange(len(case["outaged"]) + 1), ws)
        self.k0, self.k1 = int(blocks[rank][0]), int(blocks[rank][-1]) + 1
        self.h = opf_create_slice(case, self.k0, self.k1, opts, stream=stream.cuda_stream)
        self.x = opf_slice_exchange(self.h)
        self.dist, self.stream = dist, stream
        with torch.cuda.stream(stream):
            opf_slice_prime(self.h)
            self.exchange()

    def exchange(self):
        if self.dist is not None:
            self.dist.all_reduce(self.x)

    def run(self, n):
        from paper_2410_17203_gb300 import opf_slice_begin, opf_slice_finish, opf_slice_local
        opf_slice_begin(self.h, n)
        for _ in range(n):
            opf_slice_local(self.h)
            self.exchange()
            opf_slice_finish(self.h)

    def close(self):
        from paper_2410_17203_gb300 import opf_destroy
        opf_destroy(self.h)


def ours_arm(args):
    import numpy as np
    import torch

    from gridgen import case_dims, make_case
    from paper_2410_17203_gb300 import (Solver, opf_create, opf_destroy, opf_get_info, opf_iterate,
                                        opf_residuals, opf_solution)

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    # N > 1: the contingencies of one instance split over the GPUs (each rank a
    # slice, one all-reduce of the exchange buffer per iteration), unless
    # --replicas asks for an independent instance per GPU
    shard = (ws > 1 and not args.replicas) or args.shard
    case = make_case(args.config, seed=None if (ws == 1 or shard) else 1000 + rank)
    d = case_dims(case)
    B = byte_model(d)
    stream = torch.cuda.Stream(device=dev)
    opts = dict(adapt_every=10, eps=0.0)

    def barrier():
        if dist is not None:
            dist.barrier()

    if shard:
        runner = SliceRunner(case, opts, stream, dist, ws, rank)
    else:
        runner = PlainRunner(case, opts, stream)
    s = runner

    # warm-up
    with torch.cuda.stream(stream):
        runner.run(args.warmup)
    torch.cuda.synchronize()
    barrier()
    clocks = Clocks(local) if rank == 0 else None
    time.sleep(0.4 if clocks else 0.0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    with torch.cuda.stream(stream):
        runner.run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    res = opf_residuals(s.h)
    info = opf_get_info(s.h)
    kernels_per_iter = int(info["kernels_per_iteration"]) + (1 if shard else 0)   # + the exchange sums
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    # a slice run solves one instance on all GPUs; replicas solve one each
    value = (1 if shard else ws) * args.steps / (ms_max / 1e3)
    s.close()

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        Kp, L, N, S, T = d["K"] + 1, d["L"], d["N"], d["S"], d["T"]
        p_dev = np.zeros((S, T), np.float32)
        price = np.zeros((N, T), np.float32)
        h2d = sum(np.asarray(v).nbytes for k, v in case.items() if isinstance(v, np.ndarray))
        d2h = p_dev.nbytes + price.nbytes + 6 * 8
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        r2 = SliceRunner(case, opts, stream, dist, ws, rank) if shard else PlainRunner(case, opts, stream)
        with torch.cuda.stream(stream):
            r2.run(args.steps)
        r = opf_residuals(r2.h)
        opf_solution(r2.h, False, True, p_dev=p_dev, price=price)
        r2.close()
        dt = time.perf_counter() - t0
        tt = torch.tensor([dt], dtype=torch.float64, device=dev)
        if dist is not None:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e = {"value": (1 if shard else ws) * args.steps / float(tt.item()), "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "includes": "opf_create (host network upload, device arena), K iterations, "
                           "residuals + solution download, opf_destroy"}

    # the unrolled-iteration gradient, before the longer legs below
    adjoint = None
    if args.adjoint > 0 and rank == 0 and ws == 1:
        adjoint = adjoint_leg(stream, args)

    # time to the 1e-4 tolerance of Eq. (converge), adaptive penalty on: a cold
    # solve, then a load-perturbed instance solved cold and warm-started from
    # the first solution (Section 3.4)
    ttt = None
    if args.ttt and rank == 0 and ws == 1:
        ttt = time_to_tolerance(case, stream, args)
    batched = None
    if args.batched > 0 and rank == 0 and ws == 1:
        batched = batched_vs_plain(stream, args)
    learned = None
    if args.learned > 0 and rank == 0 and ws == 1:
        learned = learned_warm_start(stream, args)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        k_s = 10
        r = run_oracle(args.config, k_s, d["T"], 2, 1)
        cpu = {"value": oracle_value(r, variables_per_iter(d)), "unit": UNIT, "cores": 1, "kind": "oracle",
               "cpu": host_cpu(), "host_cores": os.cpu_count(),
               "sample": f"{args.config} network with contingencies 0..{k_s} (of {d['K']}), 2 timed "
                         f"iterations after 1 warm-up; value scaled by 4JT(K+1) variables per iteration"}
        # all host cores: the oracle sharded by contingency over single-threaded processes
        world = min(os.cpu_count() or 1, k_s + 1)
        if world > 1:
            try:
                ra = run_oracle(args.config, k_s, d["T"], 2, 1, world=world)
                cpu["all_cores"] = {"value": oracle_value(ra, variables_per_iter(d)), "unit": UNIT,
                                    "cores": world, "host_cores": os.cpu_count(),
                                    "how": "contingency shards over single-threaded processes, gloo all-reduce "
                                           "of the sums over k and the residual parts (devices evaluated by "
                                           "every process)"}
            except Exception as e:   # the single-core baseline stands on its own
                cpu["all_cores"] = {"unavailable": str(e)[:200]}

    if rank == 0:
        peak, src = peak_hbm()
        # bytes moved per GPU: a slice holds 1/ws of the contingency-replicated state
        achieved = B * args.steps / (ms / 1e3) / 1e9 / (ws if shard else 1)
        # the committed summary covers the 10k workload on one context
        traffic = profiled_traffic() if (args.config == "10k" and not shard) else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args.config, d), "N": d["N"], "L": d["L"], "T": d["T"], "K": d["K"],
                       "S": d["S"], "J": d["J"],
                       "parallelism": (f"contingency slices x{ws} (one all-reduce of the exchange buffer per iteration)"
                                       if shard else f"independent instance per GPU x{ws}"),
                       "l2": "inputs larger than L2 (state %.2f GB)" % (info["device_bytes"] / 1e9),
                       "adapt_every": 10},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": src,
                         "traffic": traffic,
                         "algorithmic_bytes_per_iteration": B,
                         "kernel": "one iteration: xs, inner, dsum, line, node and decide kernels "
                                   "replayed from CUDA graphs (unit = iteration; per-kernel shares in "
                                   "profiles/iteration_10k.txt)"},
            "variable_updates_per_s": value * variables_per_iter(d),
            "e2e": e2e,
            "gpu_launches": kernels_per_iter * args.steps + 1,   # + the call's begin kernel
            "clocks": ck,
            "residuals": [float(x) for x in res],
            "rho": [info["rho_p"], info["rho_theta"]],
        }
        if cpu:
            line["cpu_baseline"] = cpu
        if ttt:
            line["time_to_tolerance"] = ttt
        if batched:
            line["batched_vs_plain"] = batched
        if learned:
            line["learned_warm_start"] = learned
        if adjoint:
            line["adjoint"] = adjoint
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="10k")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="run the timed iterations as contingency slices even on one GPU (the default for N > 1)")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: an independent instance per GPU instead of contingency slices")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttt", dest="ttt", action="store_false",
                    help="skip the solves to eps = 1e-4 (cold, perturbed cold, perturbed warm)")
    ap.add_argument("--ttt-max", type=int, default=30000)
    ap.add_argument("--ttt-chunk", type=int, default=100)
    ap.add_argument("--ttt-alpha", type=float, default=1.5,
                    help="also solve the instance cold with this over-relaxation (1 = skip)")
    ap.add_argument("--learned", type=int, default=256,
                    help="also train the warm-start network on this many perturbed 2k instances "
                         "(a quarter, at most 64, held out) and compare iterations to eps = 1e-4: cold, learned "
                         "start, the paper's warm start (0 = skip)")
    ap.add_argument("--learned-epochs", type=int, default=40)
    ap.add_argument("--learned-lr", type=float, default=1e-3)
    ap.add_argument("--batched", type=int, default=64,
                    help="also solve this many independent instances to eps = 1e-4, one by one and as one batch "
                         "(0 = skip)")
    ap.add_argument("--stall-window", type=int, default=3000,
                    help="stall rule of the batched solves (include/opf.h opf_options.stall_window; 0 = off)")
    ap.add_argument("--adjoint", type=int, default=200,
                    help="also time the cost gradient after this many unrolled iterations on the 2k instance (0 = skip)")
    ap.add_argument("--_oracle-child", dest="oracle_child", default=None)
    args = ap.parse_args()
    if args.oracle_child:
        kw = json.loads(args.oracle_child)
        print(json.dumps(oracle_child_sharded(**kw) if "world" in kw else oracle_child(**kw)))
        return 0
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
