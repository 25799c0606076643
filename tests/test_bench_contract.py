"""bench.py's reference arm (the oracle on the host cores) keeps the JSON
contract, alone and under torchrun with two gloo ranks, where rank 0 alone
prints (CPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def lines_of(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def check_line(d, steps, warmup, n_gpus):
    assert d["impl"] == "reference"
    for k in ("metric", "unit", "dtype", "data", "scaling"):
        assert isinstance(d[k], str) and d[k]
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["steps"] == steps and d["warmup"] == warmup and d["n_gpus"] == n_gpus
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["host"]["nproc"] >= 1
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_single_process():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1", "--n", "512"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    ls = lines_of(r.stdout)
    assert len(ls) == 1
    check_line(ls[0], 2, 1, 1)


def test_reference_arm_two_ranks():
    env = dict(os.environ, GFE_BENCH_BACKEND="gloo")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", "29617", "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]  # the default 4096^2 sample (about a second)
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    ls = lines_of(r.stdout)
    assert len(ls) == 1  # rank 0 alone
    check_line(ls[0], 1, 0, 2)
