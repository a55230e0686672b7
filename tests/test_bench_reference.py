"""The reference arm of bench.py (the FP64 oracle timed on host cores), launched as two
ranks (gloo here, NCCL on GPUs): only rank 0 runs the oracle -- one complete FP64 CG
solve of the benchmark system, not extrapolated -- and prints one JSON line with the
same metric, unit and workload as the GPU arm, its own cpu_baseline and an e2e block
with no host-device traffic; the other rank exits 0 without work."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line_under_two_ranks():
    sys.path.insert(0, ROOT)
    import bench

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    env = dict(os.environ, PFMP_BENCH_GLOO="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "2", "--warmup", "1"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=1200, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["higher_is_better"] is False and d["steps"] == 2 and d["warmup"] == 1
    # value = the whole solve (the sum of the two steps), ms_per_step = the mean step
    assert d["value"] > 0 and abs(d["ms_per_step"] * 2 - d["value"]) < 1e-6 * d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "complete" in cb["sample"] and cb["cpu"]["nproc"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
