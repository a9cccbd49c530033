"""CPU: bench.py's reference arm (the FP64 oracle timed on the host cores) prints
the benchmark's JSON line, with the keys the driver reads, on a small sample;
the batch workload prints its one-line `unavailable` answer."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--impl", "reference", "--workload", "flow_p4", "--steps", "1", "--warmup", "0", "--ref-sample", "12")
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["config"]["workload"] == "flow_p4" and d["config"]["sample_n"] == 12
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_batch_is_unavailable():
    d = _run("--impl", "reference", "--workload", "batch")
    assert d["impl"] == "reference" and "unavailable" in d


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the driver launches N > 1 (torchrun, one process per rank): rank 0
    alone runs the oracle and prints; the other rank exits 0 without work."""
    import socket

    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        port = sck.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port),
                        os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0", "--ref-sample", "8", "--workload", "flow_p4"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0


def test_reference_arm_default_workload():
    """With no workload named, the reference arm times the oracle on the default
    (largest single-GPU) workload, p = 16, q = 2, g = 8, n = 2e6."""
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "0", "--ref-sample", "50")
    assert d["config"]["workload"] == "wide_p16" and d["config"]["n"] == 2_000_000
    assert d["config"]["sample_n"] == 50 and d["value"] > 0
