"""bench.py's JSON contract on the CPU: the reference arm (the oracle timed on
the host cores) prints one line with every key the contract names, and the
roofline's traffic lookup reads the committed counters."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--cpu-seconds", "0.5"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [x for x in res.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["unit"] == "Guniforms/s" and d["vs_baseline"] is None and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_traffic_lookup_reads_the_committed_counters():
    sys.path.insert(0, ROOT)
    import bench
    h = bench.source_hash(bench.KERNEL_SOURCES)  # every region marker is present
    assert len(h) == 16
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        d = json.load(f)
    for key in ("mrg_f64", "mrg_u32"):
        e = d[key]
        assert e["bytes_per_launch"] > 0 and len(e["source_hash"]) == 16 and e["captured"]
        # reported only while the kernel sources are the captured ones
        assert bench.ncu_traffic(key) == (e["bytes_per_launch"] if e["source_hash"] == h else None)
