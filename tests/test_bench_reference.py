"""The bench's reference arm on the host (no GPU): `bench.py --impl reference` times the
FP64 oracle on a bounded sample of the headline workload and prints one JSON line with
the metric, unit and direction of the GPU arm, the oracle as its CPU baseline and an
end-to-end figure with no device copies."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    sys.path.insert(0, ROOT)
    import bench
    env = dict(os.environ, OMP_NUM_THREADS="3")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    out = json.loads(lines[0])
    assert out["impl"] == "reference"
    assert out["metric"] == bench.METRIC and out["unit"] == "TFLOP/s"
    assert out["higher_is_better"] is True and out["n_gpus"] == 1
    assert out["steps"] == 1 and out["warmup"] == 0
    assert out["config"]["workload"] == "glass64_open_N262144"
    assert out["value"] > 0 and out["ms_per_step"] > 0
    cb = out["cpu_baseline"]
    # the threads the oracle ran on, not the machine's CPU count
    assert cb["kind"] == "oracle" and cb["cores"] == 3 and cb["value"] == out["value"]
    assert cb["sample"] == out["config"]["sample"]
    # the oracle parallelises over rows: at least four rows per thread keep each one busy
    r0, r1 = (int(x) for x in cb["sample"].split()[1].split(".."))
    assert r1 - r0 >= 4 * cb["cores"]
    assert "256 bins" in cb["sample"] and "64 q" in cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_two_ranks_prints_one_line():
    """Under torchrun with two ranks (gloo on the host) rank 0 alone times the oracle, on
    every CPU of the process, and prints; the other rank exits 0 without output."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), "bench.py", "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2
    # rank 0 uses every CPU of the process although the launcher sets one thread per rank
    cb = out["cpu_baseline"]
    assert cb["cores"] == len(os.sched_getaffinity(0))
    r0, r1 = (int(x) for x in cb["sample"].split()[1].split(".."))
    assert r1 - r0 >= 4 * cb["cores"]
