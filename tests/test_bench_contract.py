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


def test_clock_sampler_keeps_the_timed_window(tmp_path):
    """The clock record keeps the samples inside the timed region (a fake
    nvidia-smi log: one sample before, two inside, one after)."""
    import datetime
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    cs = bench.ClockSampler(0)
    log = tmp_path / "clocks.csv"
    log.write_text("\n".join([
        "0, 1000, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, Not Active, 2026/12/04 10:00:00.000",
        "0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active, 2026/12/04 10:00:00.100",
        "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active, 2026/12/04 10:00:00.120",
        "0, 900, 2070, 300.0, 0x8, Active, Not Active, Not Active, Not Active, 2026/12/04 10:00:01.000",
    ]) + "\n")
    cs.path = str(log)

    class FakeProc:  # stands in for the sampling process
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs.proc = FakeProc()
    t = lambda s: datetime.datetime.strptime(s, "%Y/%m/%d %H:%M:%S.%f").timestamp()
    cs.mark(t("2026/12/04 10:00:00.090"), t("2026/12/04 10:00:00.130"))
    clk = cs.stop()
    assert clk["samples"] == 2 and clk["samples_in_region"] == 2
    assert clk["sm_mhz"] == 2070.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"] and clk["power_w_max"] == 950.0
