"""bench.py's command line and the JSON line of its oracle arm (CPU only).

The oracle arm (``--impl reference``) needs no GPU; on the tiny network it
runs in seconds, so the line's keys and units are checked here.  The GPU arm
prints the same keys plus the roofline, clocks and launch count; it is run on
the GPU by the full-size tests and the benchmark itself."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*argv, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_oracle_arm_prints_one_contract_line():
    r = _bench("--impl", "reference", "--config", "tiny", "--steps", "3", "--warmup", "3")
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference"
    assert j["metric"] == "ADMM iterations/s" and j["unit"] == "iter/s"
    assert j["value"] > 0 and j["ms_per_step"] > 0
    assert (j["n_gpus"], j["steps"], j["warmup"]) == (1, 3, 3)
    assert j["higher_is_better"] is True and j["scaling"] == "weak" and j["vs_baseline"] is None
    assert j["dtype"] == "f64" and j["data"] == "synthetic"
    assert j["config"]["workload"] == "dcopf-tiny-bus-T1-K5"
    assert (j["config"]["N"], j["config"]["L"], j["config"]["T"], j["config"]["K"]) == (30, 40, 1, 5)
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == j["value"] and cb["cores"] >= 1 and cb["sample"]
    assert j["e2e"] == {"value": j["value"], "unit": "iter/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_fewer_than_three_warmup_steps_are_refused():
    r = _bench("--impl", "reference", "--config", "tiny", "--steps", "3", "--warmup", "2")
    assert r.returncode == 2 and "--warmup" in r.stderr


def test_oracle_arm_on_other_ranks_does_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--config", "tiny", "--steps", "3", "--warmup", "3"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_oracle_arm_under_torchrun_prints_one_line():
    """Launched like the multi-GPU bench (one process per rank): rank 0 alone
    times the oracle and prints; the other rank exits 0 without work."""
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", "0", os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--config", "tiny", "--steps", "3", "--warmup", "3",
                        "--gpus", "2"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["n_gpus"] == 2 and j["value"] > 0
