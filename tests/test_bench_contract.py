"""bench.py's contract on CPU: the reference arm (the oracle timed on the
host cores) prints one JSON line with the keys the harness reads, and the
committed DRAM-traffic record belongs to the current couple-lanes kernel
sources (else the bench reports no traffic)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "nodes/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "pool_200x20"


def test_traffic_record_is_used_only_for_the_kernel_sources_it_was_taken_on():
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "fsp_lanes_streamed_pool_200x20.json")))
    if rec["kernel_source_sha256_16"] != bench.kernel_source_hash():
        assert bench.read_traffic(262144) is None  # stale counters are never reported
        return
    per_node = rec["dram_bytes_per_launch"] / rec["nodes_per_launch"]
    assert abs(bench.read_traffic(262144) - per_node * 262144) < 1.0
