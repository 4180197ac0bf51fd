#!/usr/bin/env python
"""Benchmark of the bulk uniform-generation hot path on GB300.

One step = one pass of the MRG32k3a bulk workload through the C ABI:
  srng_reset (back to the start states of 2^18 streams 2^127 apart from the
  expanded seed 0x5EED5EED5EED5EED, placed by jump-ahead (K1) when the set was
  created and kept beside the working states), then srng_generate of 4096 draws
  per stream as uint32 (2^30 values), then -- after moving on -- another 4096
  draws per stream as FP64 (2^30 values).  Metric: uniforms per second
  (2^31 per step), with every output resident in HBM (12.9 GB per step,
  100x the L2, so no flush is needed between steps).

Other workloads (MRG32k3a plain 64 x 2^16 FP64, Philox4x32-10 bulk 2^30
words, the 10^4-instance batched launch with its fused Monte Carlo consumer
and the serving loop, at the offered rate and compressed 2x, 5x and 10x) are
summarised under "summary" in the same JSON line, with fractions of both the
measured copy peak and a write-only fill measured in the same run; "parity"
holds the oracle comparisons of every configuration's outputs (sampled rows,
runs, instances) and "cpu_baseline.per_config" the oracle's rate on each.
The full record (tunes, medians, the other generators) goes to the file
named by $SRNG_BENCH_DETAILS, when that is set.

--impl reference times the CPU oracle (the plain definition, OpenMP over
streams) on the host cores on a bounded sample of the same workload.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run (one process per GPU, independent replicas: rank r
holds and generates streams [r S, (r+1) S) of the sequence, a range set of
its own; no data-path collective).
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

S_STREAMS, N_DRAWS, SEED = 1 << 18, 4096, 0x5EED5EED5EED5EED
HBM_FALLBACK_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-extras", action="store_true", help="skip the other workloads")
    p.add_argument("--e2e-steps", type=int, default=8)
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="target CPU time of the oracle sample")
    p.add_argument("--case", choices=sorted(CASES), default=None,
                   help="time one kernel alone on a reduced size (for profiling), print one JSON line")
    p.add_argument("--case-scale", type=int, default=4, help="--case size = full size / this")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--case-tune", default=None,
                   help='--case launch shape as JSON, e.g. \'{"chunk": 2048, "vector_store": 3}\' (default: built-in)')
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms, each sample
    with its timestamp; started before the warm-up so that it runs through the
    whole timed region, whose samples mark() selects (all samples when the
    region is shorter than the sampling interval)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")
    window = None

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, t0: float, t1: float):
        """The timed region in host time (time.time())."""
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def when(r):
            try:
                return datetime.datetime.strptime(r[9], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except Exception:
                return None
        in_region = len(rows)
        if self.window:
            a, b = self.window
            sel = [r for r in rows if when(r) is not None and a - 0.02 <= when(r) <= b + 0.02]
            in_region = len(sel)
            if sel:
                rows = sel
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "samples_in_region": in_region,
                "power_w_max": max(pw) if pw else None}


def source_hash(parts):
    """Hash of the kernel's source: whole files, or (file, first line, last
    line) regions -- the MRG32k3a generation kernels and their dispatch, and
    the MRG32k3a device maths of the header, so that edits to the other
    generators keep the counters valid."""
    h = hashlib.sha256()
    for part in parts:
        if isinstance(part, str):
            with open(os.path.join(ROOT, part), "rb") as fh:
                h.update(fh.read())
            continue
        path, first, last = part
        with open(os.path.join(ROOT, path), "rb") as fh:
            text = fh.read()
        a = text.index(first.encode())
        b = text.index(last.encode(), a) + len(last)
        h.update(text[a:b])
    return h.hexdigest()[:16]


KERNEL_SOURCES = [
    # the MRG32k3a generation kernels with their conversions, and their launch-shape dispatch
    ("paper_1412_8266_gb300/csrc/generate.cu", "template <int GEN, int OUT>\n__device__ __forceinline__",
     "// ------------------------------------------------------------------ K3"),
    ("paper_1412_8266_gb300/csrc/generate.cu", "template <int OUT, bool VEC>\ncudaError_t mrg_dispatch_warps",
     "template <int OUT, int U, int CIPHER>"),
    # the MRG32k3a device maths and the FP32 conversion of the header
    ("include/srng_device.cuh", "namespace mrg {", "}  // namespace mrg"),
    ("include/srng_device.cuh", "__device__ __forceinline__ float to_f32(uint32_t v)", "\n}\n")]


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    sources are unchanged since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != source_hash(KERNEL_SOURCES):
        return None
    return e.get("bytes_per_launch")


# --------------------------------------------------------------------- CPU oracle
def host_threads() -> int:
    """Host cores this process may run on (the oracle's thread count)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_sample(target_s: float, threads: int = 0):
    """Time the oracle on a bounded sample of the MRG32k3a bulk workload:
    the first s streams of the same set, 4096 draws each as uint32, then 4096
    more as FP64 (the shape of one step), s chosen so the run takes about
    target_s seconds, on `threads` host threads (0: all).  Returns
    (Guniforms/s, cores used, description)."""
    from oracle import oracle as O
    y0 = O.seed_expand(SEED)
    threads = threads or host_threads()

    def run(s):
        starts = O.mrg_stream_starts(y0, 127, 0, s)
        t0 = time.perf_counter()
        _, st = O.mrg_bulk(starts, N_DRAWS, O.OUT_U32, threads)
        O.mrg_bulk(st, N_DRAWS, O.OUT_F64, threads)
        return time.perf_counter() - t0

    probe = 64 * threads
    dt = run(probe)
    s = int(min(S_STREAMS, max(probe, probe * target_s / max(dt, 1e-6))))
    dt = run(s)
    nums = 2 * s * N_DRAWS
    return nums / dt / 1e9, threads, (f"{s} of {S_STREAMS} streams x {N_DRAWS} draws, uint32 then FP64 "
                                      f"({nums} values in {dt:.1f} s on {threads} threads)")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    vals = []
    cores = 0
    desc = ""
    for _ in range(args.warmup):
        oracle_sample(args.cpu_seconds / 4)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, cores, desc = oracle_sample(args.cpu_seconds / max(1, args.steps))
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": "Guniforms/s (MRG32k3a bulk, uint32 + FP64, bit-exact)", "value": value,
        "unit": "Guniforms/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "MRG32k3a bulk: 2^18 streams x 4096 draws, uint32 + FP64 (CPU sample)",
                   "streams": S_STREAMS, "draws_per_stream": N_DRAWS, "seed": hex(SEED)},
        "cpu_baseline": {"value": value, "unit": "Guniforms/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "Guniforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1412_8266_gb300 as srng
    from paper_1412_8266_gb300 import autotune
    from paper_1412_8266_gb300.replicas import max_over_ranks, stream_range

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = measured_peaks()

    # launch shapes for this workload, chosen by timing (outputs do not depend on them)
    t_tune = time.perf_counter()
    tune_u, _ = autotune.tune_generate(srng.SRNG_MRG32K3A, srng.SRNG_OUT_U32, S_STREAMS, N_DRAWS, use_cache=False,
                                       install=False)
    tune_f, _ = autotune.tune_generate(srng.SRNG_MRG32K3A, srng.SRNG_OUT_F64, S_STREAMS, N_DRAWS, use_cache=False,
                                       install=False)
    t_tune = time.perf_counter() - t_tune

    # replicas: rank r holds and generates streams [r S, (r+1) S) of one sequence
    base, _ = stream_range(rank, world, S_STREAMS)
    h = srng.srng_create_range(srng.SRNG_MRG32K3A, SEED, base, S_STREAMS, srng.SRNG_SPACING_STREAM, None, stream)
    b = 0
    out_u = torch.empty(S_STREAMS * N_DRAWS, dtype=torch.int32, device=dev)
    out_f = torch.empty(S_STREAMS * N_DRAWS, dtype=torch.float64, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]

    def step(k=None):
        srng.srng_reset(h, stream)
        if k is not None:
            ev[k][0].record(stream)
        srng.srng_generate_tuned(h, b, S_STREAMS, N_DRAWS, srng.SRNG_OUT_U32, out_u, tune_u, stream)
        if k is not None:
            ev[k][1].record(stream)
            ev[k][2].record(stream)
        srng.srng_generate_tuned(h, b, S_STREAMS, N_DRAWS, srng.SRNG_OUT_F64, out_f, tune_f, stream)
        if k is not None:
            ev[k][3].record(stream)

    clocks = ClockSampler(local)
    clocks.start()  # running before the timed region starts
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    host_t0 = time.time()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(k)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark(host_t0, time.time())
    clk = clocks.stop()
    ms_total = max_over_ranks(t_start.elapsed_time(t_end), dev)
    ms_step = ms_total / args.steps
    numbers = 2 * S_STREAMS * N_DRAWS
    value = world * numbers / (ms_step / 1e3) / 1e9
    ms_u = statistics.mean(ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps))
    ms_f = statistics.mean(ev[k][2].elapsed_time(ev[k][3]) for k in range(args.steps))
    bytes_u, bytes_f = S_STREAMS * N_DRAWS * 4, S_STREAMS * N_DRAWS * 8
    dom = "mrg_f64" if ms_f * 1 >= ms_u else "mrg_u32"
    dom_bytes, dom_ms = (bytes_f, ms_f) if dom == "mrg_f64" else (bytes_u, ms_u)
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9

    # end to end through the host-buffer entry point (device -> pinned host inside the timed region)
    e2e = None
    if True:
        host_u = torch.empty(S_STREAMS * N_DRAWS, dtype=torch.int32, pin_memory=True)
        host_f = torch.empty(S_STREAMS * N_DRAWS, dtype=torch.float64, pin_memory=True)

        def e2e_step():
            srng.srng_reset(h, stream)  # generation into pinned host memory (see srng_generate_host)
            srng.srng_generate_host(h, b, S_STREAMS, N_DRAWS, srng.SRNG_OUT_U32, host_u, stream)
            srng.srng_generate_host(h, b, S_STREAMS, N_DRAWS, srng.SRNG_OUT_F64, host_f, stream)

        for _ in range(2):  # untimed: the first passes over fresh host buffers can stall
            e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        each = []
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            t1 = time.perf_counter()
            e2e_step()  # srng_generate_host synchronises the stream before returning
            each.append(time.perf_counter() - t1)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dev)
        # the host copy must equal the device output of the same step
        same = bool(np.array_equal(host_u[:1 << 20].numpy(), out_u[:1 << 20].cpu().numpy()))
        # the host link alone: one 1 GiB device -> pinned host copy (best of 3)
        src = torch.empty(1 << 28, dtype=torch.float32, device=dev)
        dst = torch.empty(1 << 28, dtype=torch.float32, pin_memory=True)
        link_ms, _ = _time(torch, stream, lambda: dst.copy_(src, non_blocking=True), reps=3, warm=1)
        link = (1 << 30) / link_ms / 1e6
        del src, dst
        e2e_gbs = (bytes_u + bytes_f) / e2e_s / 1e9
        e2e = {"value": world * numbers / e2e_s / 1e9, "unit": "Guniforms/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": bytes_u + bytes_f, "ms_per_step": e2e_s * 1e3,
               "ms_each_step": [round(x * 1e3, 2) for x in each], "matches_device_output": same,
               "GB_s": e2e_gbs, "host_link_GB_s": link, "frac_of_host_link": e2e_gbs / link,
               "bound": "host link (device -> pinned host copy measured in this run)"}
        del host_u, host_f

    # parity of the timed step's outputs: sampled streams (rows) of both outputs
    # against the oracle, from the seed alone
    par_c2 = parity_c2(out_u, out_f, S_STREAMS, base) if rank == 0 else {}
    srng.srng_destroy(h)
    del out_u, out_f
    torch.cuda.empty_cache()

    wfill = write_only_peak(torch, dev, stream)
    c2 = {"ms_u32": ms_u, "ms_f64": ms_f, "Guniforms_s": value / world,
          "frac_copy": {"u32": bytes_u / ms_u / 1e6 / peak, "f64": bytes_f / ms_f / 1e6 / peak},
          "frac_write_fill": {"u32": bytes_u / ms_u / 1e6 / wfill["GB_s"], "f64": bytes_f / ms_f / 1e6 / wfill["GB_s"]},
          "parity": par_c2}
    line = {
        "metric": "Guniforms/s (MRG32k3a bulk, uint32 + FP64, bit-exact)", "value": value, "unit": "Guniforms/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": "MRG32k3a bulk: 2^18 streams x 4096 draws, uint32 + FP64 per step",
                   "streams_per_gpu": S_STREAMS, "draws_per_stream": N_DRAWS, "seed": hex(SEED),
                   "spacing": "2^127", "outputs_bytes_per_step": bytes_u + bytes_f,
                   "l2": "no flush: 12.9 GB of outputs per step, 100x the L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "traffic": ncu_traffic(dom), "algorithmic_bytes_per_launch": dom_bytes,
                     "ms_per_launch": dom_ms, "write_fill_GB_s": wfill["GB_s"],
                     "frac_of_write_fill": achieved / wfill["GB_s"]},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": 4 * args.steps,  # per step: generate + state advance, twice (the reset is a device copy)
        "parity": {"C2": par_c2},
    }
    details = {"kernels": {"mrg_u32": {"ms": ms_u}, "mrg_f64": {"ms": ms_f}},
               "tune": {"mrg_u32": tune_u, "mrg_f64": tune_f, "tuning_s": t_tune}, "write_only_fill": wfill}
    summary = {"C2": c2}
    if rank == 0:
        cpu = {}
        v, cores, desc = oracle_sample(args.cpu_seconds)
        v1, _, desc1 = oracle_sample(args.cpu_seconds / 4, threads=1)
        if not args.no_extras:
            try:
                summ, det, par, cpu = extras(torch, srng, dev, stream, peak, wfill["GB_s"], args.cpu_seconds)
                summary.update(summ)
                details["workloads"] = det
                line["parity"].update(par)
            except Exception as ex:  # report, do not hide
                summary["error"] = repr(ex)
        line["cpu_baseline"] = {"value": v, "unit": "Guniforms/s", "cores": cores, "kind": "oracle", "sample": desc,
                                "single_core": {"value": v1, "sample": desc1}, "per_config": cpu}
        line["parity"]["mismatches"] = sum(int(p.get("mismatches", 0)) for p in line["parity"].values()
                                           if isinstance(p, dict))
        line["summary"] = summary
        write_details(details)
        print(json.dumps(_rounded(line), separators=(",", ":")), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _rounded(x, nd=4):
    """Floats to nd significant digits, so the one JSON line stays short."""
    if isinstance(x, float):
        return float(f"{x:.{nd}g}")
    if isinstance(x, dict):
        return {k: _rounded(v, nd) for k, v in x.items()}
    if isinstance(x, list):
        return [_rounded(v, nd) for v in x]
    return x


def write_details(details):
    """The long per-workload record (tunes, every timing) goes to a file, not
    into the one JSON line: the one $SRNG_BENCH_DETAILS names, else nowhere."""
    path = os.environ.get("SRNG_BENCH_DETAILS")
    if path:
        with open(path, "w") as f:
            json.dump(details, f, indent=1)


def parity_c2(out_u, out_f, n_streams, base, rows=48):
    """Sampled rows of the bulk step's outputs against the oracle: stream s's
    first 4096 draws as uint32, then its next 4096 as FP64."""
    import numpy as np
    from oracle import oracle as O
    if not n_streams:
        return {"rows": 0}
    rng = np.random.default_rng(1412)
    pick = sorted(set([0, n_streams - 1] + rng.integers(0, n_streams, rows - 2).tolist()))
    y0 = O.seed_expand(SEED)
    bad = 0
    gu = out_u.view(-1, N_DRAWS)
    gf = out_f.view(-1, N_DRAWS)
    for s in pick:
        st = O.mrg_stream_starts(y0, 127, base + s, 1)[0]
        ru, st = O.mrg_generate(st, N_DRAWS, O.OUT_U32)
        rf, _ = O.mrg_generate(st, N_DRAWS, O.OUT_F64)
        bad += int(np.count_nonzero(gu[s].cpu().numpy().view(np.uint32) != ru))
        bad += int(np.count_nonzero(gf[s].cpu().numpy().view(np.uint64) != rf.view(np.uint64)))
    return {"rows": len(pick), "values": 2 * len(pick) * N_DRAWS, "mismatches": bad}


def _time(torch, stream, fn, reps=5, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return min(ts), statistics.median(ts)


def write_only_peak(torch, dev, stream):
    """Context for the write-bound kernels: HBM write-only bandwidth of a plain
    device fill (torch's zero_ on 8 GiB, best of 5) next to the measured copy peak."""
    buf = torch.empty(1 << 31, dtype=torch.float32, device=dev)
    best, med = _time(torch, stream, lambda: buf.zero_(), reps=5, warm=2)
    del buf
    torch.cuda.empty_cache()
    return {"GB_s": (8 << 30) / best / 1e6, "ms_best": best, "how": "torch zero_ of 8 GiB, best of 5"}


def _threaded(fn, jobs, threads):
    """Run fn over jobs on host threads (the oracle's C calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(fn, jobs))


def _fracs(nbytes, ms, peak, wfill):
    gbs = nbytes / ms / 1e6
    return {"GB_s": gbs, "frac_copy": gbs / peak, "frac_write_fill": gbs / wfill}


def extras(torch, srng, dev, stream, peak, wfill, cpu_seconds):
    """The other workloads.  Returns (summary, details, parity, cpu): a short
    per-configuration summary for the JSON line, the full record for the
    details file, the oracle comparisons, and the oracle's timings on each
    configuration (a bounded sample, on all host threads)."""
    import numpy as np
    from oracle import oracle as O
    from paper_1412_8266_gb300 import autotune
    from paper_1412_8266_gb300 import workload as W
    threads = host_threads()
    summ, det, par, cpu = {}, {}, {}, {}

    # ---- C1: MRG32k3a plain, 64 streams x 2^16 FP64 (all-12345 state, 2^127 apart)
    h = srng.srng_create_from_state([12345] * 6, 64, srng.SRNG_SPACING_STREAM, stream)
    o = torch.empty(64 << 16, dtype=torch.float64, device=dev)
    call = lambda s: (srng.srng_reset(h, s), srng.srng_generate(h, 0, 64, 1 << 16, srng.SRNG_OUT_F64, o, s))
    best, med = _time(torch, stream, lambda: call(stream))
    # the same call captured 20 times in a CUDA graph: device time per call, without host launch gaps
    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        call(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        for _ in range(20):
            call(side)
    gb, gm = _time(torch, stream, g.replay)
    # the generation call alone (kernel + state advance), 20 calls per graph: the streams move on
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=side):
        for _ in range(20):
            srng.srng_generate(h, 0, 64, 1 << 16, srng.SRNG_OUT_F64, o, side)
    gg, _ = _time(torch, stream, g2.replay)
    del g2
    # the state advance alone (the call's second, dependent launch), 20 per graph
    g3 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g3, stream=side):
        for _ in range(20):
            srng.srng_jump(h, 0, 64, srng.SRNG_JUMP_DRAWS, 1 << 16, side)
    ga, _ = _time(torch, stream, g3.replay)
    del g3
    call(stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref, _ = O.mrg_bulk(O.mrg_stream_starts([12345] * 6, 127, 0, 64), 1 << 16, O.OUT_F64, threads)
    t_or = time.perf_counter() - t0
    bad = int(np.count_nonzero(o.cpu().numpy().view(np.uint64) != ref.ravel().view(np.uint64)))
    par["C1"] = {"values": 64 << 16, "mismatches": bad}
    cpu["C1"] = {"Guniforms_s": (64 << 16) / t_or / 1e9, "cores": threads, "sample": "whole workload"}
    us = gb / 20 * 1e3
    summ["C1"] = {"us_per_call_graph": us, "us_per_call_plain": best * 1e3, "us_per_generate_graph": gg / 20 * 1e3,
                  "us_per_advance_graph": ga / 20 * 1e3,
                  "Guniforms_s": (64 << 16) / us / 1e3, **_fracs((64 << 16) * 8, us / 1e3, peak, wfill)}
    det["mrg_plain_64x65536_f64"] = {"plain_ms_best": best, "plain_ms_median": med, "graph_20_calls_ms": gb}
    del g, o
    srng.srng_destroy(h)

    # ---- C3: Philox bulk, 2^30 words of one stream, u32 and f32
    n = 1 << 30
    key = (0xC0FFEE, 0)
    ph = {}
    tunes = {}
    h = srng.srng_create(srng.SRNG_PHILOX4X32_10, 0xC0FFEE, 1, srng.SRNG_SPACING_STREAM, stream)
    rng = np.random.default_rng(3)
    pos = sorted(set([0, n - (1 << 16)] + (rng.integers(0, n >> 16, 30) << 16).tolist()))
    c3 = {}
    bad = 0
    for name, t, dt in (("u32", srng.SRNG_OUT_U32, torch.int32), ("f32", srng.SRNG_OUT_F32, torch.float32)):
        tunes[t] = autotune.tune_generate(srng.SRNG_PHILOX4X32_10, t, 1, n, use_cache=False, install=False)[0]
        o = torch.empty(n, dtype=dt, device=dev)
        best, med = _time(torch, stream, lambda: (srng.srng_reset(h, stream),
                                                  srng.srng_generate_tuned(h, 0, 1, n, t, o, tunes[t], stream)))
        ph[name] = {"ms_best": best, "ms_median": med, "tune": tunes[t]}
        c3["ms_" + name] = best
        c3[name] = _fracs(n * 4, best, peak, wfill)
        t0 = time.perf_counter()
        refs = _threaded(lambda p: O.philox_generate(key, 0, p, 1 << 16, t), pos, threads)
        t_or = time.perf_counter() - t0
        for p, r in zip(pos, refs):
            bad += int(np.count_nonzero(o[p:p + (1 << 16)].cpu().numpy().view(np.uint32) != r.view(np.uint32)))
        cpu["C3_" + name] = {"Guniforms_s": len(pos) * (1 << 16) / t_or / 1e9, "cores": threads,
                             "sample": f"{len(pos)} runs of 2^16 words at seeded positions"}
        del o
    par["C3"] = {"values": 2 * len(pos) * (1 << 16), "mismatches": bad}
    summ["C3"] = c3
    det["philox_bulk_2^30"] = ph
    # variates: 2^30 FP32 Philox uniforms -> exponential / normal, and fused into generation
    u = torch.empty(n, dtype=torch.float32, device=dev)
    srng.srng_reset(h, stream)
    srng.srng_generate_tuned(h, 0, 1, n, srng.SRNG_OUT_F32, u, tunes[srng.SRNG_OUT_F32], stream)
    z = torch.empty_like(u)
    var = {}
    for name, d in (("exponential", srng.SRNG_DIST_EXPONENTIAL), ("normal", srng.SRNG_DIST_NORMAL)):
        best, med = _time(torch, stream, lambda: srng.srng_transform(d, u, n, z, stream))
        var[name] = {"ms_best": best, **_fracs(n * 8, best, peak, wfill)}
    for name, t in (("fused_exponential", srng.SRNG_OUT_EXP_F32), ("fused_normal", srng.SRNG_OUT_NORMAL_F32)):
        tt = autotune.tune_generate(srng.SRNG_PHILOX4X32_10, t, 1, n, use_cache=False, install=False)[0]
        best, med = _time(torch, stream, lambda: (srng.srng_reset(h, stream),
                                                  srng.srng_generate_tuned(h, 0, 1, n, t, z, tt, stream)))
        var[name] = {"ms_best": best, "Gvariates_s": n / best / 1e6, "tune": tt,
                     "vs_generate_then_transform": (c3["ms_f32"] + var[name[6:]]["ms_best"]) / best}
    del u, z
    srng.srng_destroy(h)
    det["variates_2^30_f32"] = var
    summ["variates"] = {k: round(v["ms_best"], 4) for k, v in var.items()}
    # Threefry (both word sizes) and TinyMT32 bulk: the rows beyond the first hot path
    for key_name, gen in (("threefry_bulk_2^30", srng.SRNG_THREEFRY4X32_20),
                          ("threefry4x64_bulk_2^30", srng.SRNG_THREEFRY4X64_20)):
        tf = {}
        h = srng.srng_create(gen, 0xC0FFEE, 1, srng.SRNG_SPACING_STREAM, stream)
        for name, t, dt in (("u32", srng.SRNG_OUT_U32, torch.int32), ("f32", srng.SRNG_OUT_F32, torch.float32)):
            tt = autotune.tune_generate(gen, t, 1, n, use_cache=False, install=False)[0]
            o = torch.empty(n, dtype=dt, device=dev)
            best, med = _time(torch, stream, lambda: (srng.srng_reset(h, stream),
                                                      srng.srng_generate_tuned(h, 0, 1, n, t, o, tt, stream)))
            tf[name] = {"ms_best": best, "tune": tt, **_fracs(n * 4, best, peak, wfill)}
            del o
        srng.srng_destroy(h)
        det[key_name] = tf
    tm = {}
    h = srng.srng_create(srng.SRNG_TINYMT32, SEED, S_STREAMS, srng.SRNG_SPACING_STREAM, stream)
    for name, t, dt in (("u32", srng.SRNG_OUT_U32, torch.int32), ("f64", srng.SRNG_OUT_F64, torch.float64)):
        o = torch.empty(S_STREAMS * N_DRAWS, dtype=dt, device=dev)
        best, med = _time(torch, stream, lambda: srng.srng_generate(h, 0, S_STREAMS, N_DRAWS, t, o, stream))
        tm[name] = {"ms_best": best, **_fracs(o.numel() * o.element_size(), best, peak, wfill)}
        del o
    srng.srng_destroy(h)
    det["tinymt_bulk_2^18x4096"] = tm
    lay = {}
    o = torch.empty(S_STREAMS * N_DRAWS, dtype=torch.int32, device=dev)
    for name, gen in (("counter_split", srng.SRNG_PHILOX4X32_10), ("keyed", srng.SRNG_PHILOX4X32_10_KEYED)):
        h = srng.srng_create(gen, 0xC0FFEE, S_STREAMS, srng.SRNG_SPACING_STREAM, stream)
        best, med = _time(torch, stream, lambda: (srng.srng_reset(h, stream),
                                                  srng.srng_generate_tuned(h, 0, S_STREAMS, N_DRAWS, srng.SRNG_OUT_U32,
                                                                           o, tunes[srng.SRNG_OUT_U32], stream)))
        lay[name] = {"ms_best": best, **_fracs(o.numel() * 4, best, peak, wfill)}
        srng.srng_destroy(h)
    del o
    det["philox_layouts_2^18x4096_u32"] = lay
    summ["beyond"] = {"threefry4x32_u32_frac_copy": det["threefry_bulk_2^30"]["u32"]["frac_copy"],
                      "threefry4x64_u32_frac_copy": det["threefry4x64_bulk_2^30"]["u32"]["frac_copy"],
                      "tinymt_u32_frac_copy": tm["u32"]["frac_copy"], "tinymt_f64_frac_copy": tm["f64"]["frac_copy"],
                      "philox_keyed_frac_copy": lay["keyed"]["frac_copy"]}

    # ---- C4: batched uneven, 10^4 instances: one graph launch vs one launch per instance; fused pi
    gens, lengths, outoff = W.batched_instances()
    ni = len(gens)
    total = int(outoff[-1] + lengths[-1])
    hm = srng.srng_create(srng.SRNG_MRG32K3A, SEED, ni, srng.SRNG_SPACING_STREAM, stream)
    hp = srng.srng_create(srng.SRNG_PHILOX4X32_10, 0xC0FFEE, ni, srng.SRNG_SPACING_STREAM, stream)
    inst = [srng.Instance(set_index=int(gens[i]), stream=i, offset=0, length=int(lengths[i]),
                          out_offset=int(outoff[i])) for i in range(ni)]
    out = torch.empty(total, dtype=torch.int32, device=dev)
    btune, _ = autotune.tune_batch([hm, hp], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, out, reps=2)
    plan = srng.srng_batch_plan_create([hm, hp], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, out, btune, stream)
    bb, bm = _time(torch, stream, lambda: srng.srng_batch_plan_launch(plan, stream), reps=5)
    items, _ = srng.srng_batch_plan_info(plan)
    srng.srng_batch_plan_destroy(plan)
    # oracle on a seeded sample of instances (also the parity check of the batched output)
    draws = int(np.sum(lengths))
    rng = np.random.default_rng(9)
    order = rng.permutation(ni)
    pick, acc = [], 0
    for i in order:
        if acc > draws // 40:
            break
        pick.append(int(i))
        acc += int(lengths[i])
    pick = sorted(pick)
    pl = np.array([int(lengths[i]) for i in pick], dtype=np.uint64)
    po = np.zeros(len(pick), dtype=np.uint64)
    po[1:] = np.cumsum(pl[:-1])
    y0 = O.seed_expand(SEED)
    mst = np.stack([O.mrg_stream_starts(y0, 127, i, 1)[0] for i in pick])
    pg = np.array([int(gens[i]) for i in pick], dtype=np.int32)
    t0 = time.perf_counter()
    ref = O.batch(pg, mst, (0xC0FFEE, 0), pick, np.zeros(len(pick), dtype=np.uint64), pl, po, 0, O.OUT_U32,
                  total=int(pl.sum()), threads=threads)
    t_or = time.perf_counter() - t0
    bad = 0
    for j, i in enumerate(pick):
        L, off = int(lengths[i]), int(outoff[i])
        bad += int(np.count_nonzero(out[off:off + L].cpu().numpy().view(np.uint32) != ref[int(po[j]):int(po[j]) + L]))
    views = [out[int(outoff[i]):int(outoff[i]) + int(lengths[i])] for i in range(ni)]

    def plain():
        for i in range(ni):
            srng.srng_generate(hm if gens[i] == 0 else hp, i, 1, int(lengths[i]), srng.SRNG_OUT_U32, views[i], stream)

    pb, pm = _time(torch, stream, plain, reps=2, warm=1)
    srng.srng_reset(hm, stream)  # the plain launches moved the streams on; the fused plan starts from the start
    srng.srng_reset(hp, stream)
    counts = torch.empty(ni, dtype=torch.int64, device=dev)
    ptune, _ = autotune.tune_batch([hm, hp], inst, srng.SRNG_BATCH_FUSED_PI, srng.SRNG_OUT_U32, counts, reps=2)
    plan = srng.srng_batch_plan_create([hm, hp], inst, srng.SRNG_BATCH_FUSED_PI, srng.SRNG_OUT_U32, counts, ptune,
                                       stream)
    fb, fm = _time(torch, stream, lambda: srng.srng_batch_plan_launch(plan, stream), reps=5)
    srng.srng_batch_plan_destroy(plan)
    c = counts.cpu().numpy()
    t0 = time.perf_counter()
    refc = O.batch(pg, mst, (0xC0FFEE, 0), pick, np.zeros(len(pick), dtype=np.uint64), pl, po, 1, O.OUT_U32,
                   threads=threads)
    t_orc = time.perf_counter() - t0
    badc = int(np.count_nonzero(np.array([c[i] for i in pick]) != refc))
    par["C4"] = {"instances": len(pick), "values": int(pl.sum()), "counts": len(pick), "mismatches": bad + badc}
    cpu["C4"] = {"Guniforms_s": int(pl.sum()) / t_or / 1e9, "fused_pi_Guniforms_s": int(pl.sum()) / t_orc / 1e9,
                 "cores": threads, "sample": f"{len(pick)} of {ni} instances ({int(pl.sum())} draws)"}
    pairs = int(np.sum(lengths // 2))
    summ["C4"] = {"batched_ms": bb, "plain_ms": pb, "speedup": pb / bb, "fused_pi_ms": fb,
                  "Guniforms_s": draws / bb / 1e6, **_fracs(draws * 4, bb, peak, wfill),
                  "pi": 4.0 * c.sum() / pairs}
    det["batched_10k_u32"] = {"draws": draws, "work_items": items, "batched_ms": bb, "batched_ms_median": bm,
                              "plain_per_instance_ms": pb, "plain_launches": 2 * ni, "fused_pi_ms": fb,
                              "tune_write": btune, "tune_fused_pi": ptune}
    srng.srng_destroy(hm)
    srng.srng_destroy(hp)
    del out, views, counts
    torch.cuda.empty_cache()

    # ---- C5: serving
    sv, cpu5 = serving(srng, threads, cpu_seconds)
    det["serving"] = sv
    cpu["C5"] = cpu5
    b1, p1 = sv["rates"]["1x"]["batched"], sv["rates"]["1x"]["plain"]
    summ["C5"] = {"offered_Guniforms_s": sv["offered_Guniforms_s"], "requests": sv["requests"],
                  "batched": {"Guniforms_s": b1["Guniforms_s"], "p50_us": b1["p50_us"], "p99_us": b1["p99_us"]},
                  "plain": {"Guniforms_s": p1["Guniforms_s"], "p50_us": p1["p50_us"], "p99_us": p1["p99_us"]},
                  "capacity_Guniforms_s": {k: {"batched": v["batched"]["Guniforms_s"], "plain": v["plain"]["Guniforms_s"],
                                               "batched_p99_us": v["batched"]["p99_us"]}
                                           for k, v in sv["rates"].items() if k != "1x"}}
    return summ, det, par, cpu


def serving(srng, threads, cpu_seconds, seconds=1.0):
    """Serving workload: Poisson arrivals (20k/s) of FP32 requests, n log-uniform
    in [1e3, 1e8], over 10^6 MRG32k3a substreams, 16 GB output budget, replayed
    by the library's native client; continuous batching vs one request per
    step with one step in flight (plain per-request launches), at the offered
    rate and at 2x, 5x and 10x it (the same requests, arrivals compressed),
    which shows each form's capacity.  Also the oracle's rate on a sample of
    the same requests (jump to the request's position, then step)."""
    import numpy as np
    from oracle import oracle as O
    from paper_1412_8266_gb300 import workload as W
    trace = [(r.arrival_s, r.stream, r.n) for r in W.serving_trace(seconds)]
    h = srng.srng_create_from_state([12345] * 6, W.SERVING["n_streams"], srng.SRNG_SPACING_SUBSTREAM)
    out = {"requests": len(trace), "draws": sum(r[2] for r in trace), "arrival_s": seconds,
           "offered_Guniforms_s": sum(r[2] for r in trace) / seconds / 1e9, "rates": {}}
    try:
        for k in (1, 2, 5, 10):
            res = {}
            for name, cfg in (("batched", dict(budget_bytes=W.SERVING["budget"])),
                              ("plain", dict(budget_bytes=W.SERVING["budget"], max_inflight=1, max_step_requests=1))):
                srv = srng.srng_server_create(h, cfg)
                try:
                    srng.srng_server_replay(srv, trace[:200], srng.SRNG_OUT_F32, 0.0)  # warm-up
                    st = srng.srng_server_replay(srv, trace, srng.SRNG_OUT_F32, 1.0 / k, 600000)
                finally:
                    srng.srng_server_destroy(srv)
                res[name] = {"p50_us": st.p50_us, "p99_us": st.p99_us, "mean_us": st.mean_us, "max_us": st.max_us,
                             "wall_s": st.wall_s,
                             "Guniforms_s": st.draws_completed / st.wall_s / 1e9 if st.wall_s else None,
                             "completed": st.completed, "steps": st.steps, "kernels": st.kernels,
                             "peak_pool_GB": st.peak_pool_bytes / 1e9}
            out["rates"][f"{k}x"] = res
    finally:
        srng.srng_destroy(h)
    # the oracle on a sample of the same requests
    rng = np.random.default_rng(5)
    idx = rng.permutation(len(trace))
    sample, acc = [], 0
    budget = int(150e6 * max(1.0, cpu_seconds / 10.0) * threads / 16)
    for i in idx:
        if acc >= budget:
            break
        sample.append(trace[int(i)])
        acc += trace[int(i)][2]

    def one(r):
        st = O.mrg_stream_starts([12345] * 6, 76, r[1], 1)[0]
        v, _ = O.mrg_generate(st, r[2], O.OUT_F32)
        return v.size

    t0 = time.perf_counter()
    done = sum(_threaded(one, sample, threads))
    dt = time.perf_counter() - t0
    return out, {"Guniforms_s": done / dt / 1e9, "cores": threads,
                 "sample": f"{len(sample)} of {len(trace)} requests ({done} draws), each from its substream start"}


def run_case(args):
    """One workload's kernel alone, args.reps launches, at full size / scale."""
    import torch

    import paper_1412_8266_gb300 as srng
    from paper_1412_8266_gb300 import workload as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream(dev)
    c = args.case
    k = max(1, args.case_scale)
    res = {"case": c, "scale": k, "tune": args.case_tune}
    if c.startswith("mrg") and c != "mrg_plain":
        S = S_STREAMS // k
        t = srng.SRNG_OUT_U32 if c == "mrg_u32" else srng.SRNG_OUT_F64
        h = srng.srng_create(srng.SRNG_MRG32K3A, SEED, S, srng.SRNG_SPACING_STREAM, stream)
        o = torch.empty(S * N_DRAWS, dtype=torch.int32 if t == 0 else torch.float64, device=dev)
        tune = json.loads(args.case_tune) if args.case_tune else None
        fn = lambda: srng.srng_generate_tuned(h, 0, S, N_DRAWS, t, o, tune, stream)
        nbytes, nvals = o.numel() * o.element_size(), o.numel()
    elif c in ("philox_many_u32", "philox_keyed_many_u32"):
        g = srng.SRNG_PHILOX4X32_10 if c == "philox_many_u32" else srng.SRNG_PHILOX4X32_10_KEYED
        S = S_STREAMS // k
        h = srng.srng_create(g, 0xC0FFEE, S, srng.SRNG_SPACING_STREAM, stream)
        o = torch.empty(S * N_DRAWS, dtype=torch.int32, device=dev)
        tune = json.loads(args.case_tune) if args.case_tune else None
        fn = lambda: srng.srng_generate_tuned(h, 0, S, N_DRAWS, srng.SRNG_OUT_U32, o, tune, stream)
        nbytes, nvals = o.numel() * 4, o.numel()
    elif c.startswith("philox") or c.startswith("threefry"):
        n = (1 << 30) // k
        t = {"u32": srng.SRNG_OUT_U32, "f32": srng.SRNG_OUT_F32, "f64": srng.SRNG_OUT_F64,
             "normal": srng.SRNG_OUT_NORMAL_F32}[c.split("_")[1]]
        g = (srng.SRNG_PHILOX4X32_10 if c.startswith("philox") else
             srng.SRNG_THREEFRY4X64_20 if c.startswith("threefry64") else srng.SRNG_THREEFRY4X32_20)
        h = srng.srng_create(g, 0xC0FFEE, 1, srng.SRNG_SPACING_STREAM, stream)
        dt = torch.int32 if t == 0 else torch.float64 if t == srng.SRNG_OUT_F64 else torch.float32
        o = torch.empty(n, dtype=dt, device=dev)
        tune = json.loads(args.case_tune) if args.case_tune else None
        fn = lambda: srng.srng_generate_tuned(h, 0, 1, n, t, o, tune, stream)
        nbytes, nvals = n * o.element_size(), n
    elif c == "mrg_plain":
        # 64 streams x 2^16 FP64 from the all-12345 state, 2^127 apart (the whole workload; no scaling)
        h = srng.srng_create_from_state([12345] * 6, 64, srng.SRNG_SPACING_STREAM, stream)
        o = torch.empty(64 << 16, dtype=torch.float64, device=dev)
        tune = json.loads(args.case_tune) if args.case_tune else None
        fn = lambda: srng.srng_generate_tuned(h, 0, 64, 1 << 16, srng.SRNG_OUT_F64, o, tune, stream)
        nbytes, nvals = o.numel() * 8, o.numel()
    elif c.startswith("tinymt"):
        S = S_STREAMS // k
        t = srng.SRNG_OUT_U32 if c == "tinymt_u32" else srng.SRNG_OUT_F64
        h = srng.srng_create(srng.SRNG_TINYMT32, SEED, S, srng.SRNG_SPACING_STREAM, stream)
        o = torch.empty(S * N_DRAWS, dtype=torch.int32 if t == 0 else torch.float64, device=dev)
        tune = json.loads(args.case_tune) if args.case_tune else None
        fn = lambda: srng.srng_generate_tuned(h, 0, S, N_DRAWS, t, o, tune, stream)
        nbytes, nvals = o.numel() * o.element_size(), o.numel()
    elif c == "serving":
        # the serving trace replayed once at its offered rate through the default server
        from paper_1412_8266_gb300 import workload as W
        trace = [(r.arrival_s, r.stream, r.n) for r in W.serving_trace(1.0)]
        h = srng.srng_create_from_state([12345] * 6, W.SERVING["n_streams"], srng.SRNG_SPACING_SUBSTREAM, stream)
        srv = srng.srng_server_create(h, dict(budget_bytes=W.SERVING["budget"]))
        try:
            srng.srng_server_replay(srv, trace[:200], srng.SRNG_OUT_F32, 0.0)  # warm-up
            st = srng.srng_server_replay(srv, trace, srng.SRNG_OUT_F32, 1.0, 600000)
        finally:
            srng.srng_server_destroy(srv)
            srng.srng_destroy(h)
        res.update({"requests": len(trace), "steps": st.steps, "kernels": st.kernels, "p50_us": st.p50_us,
                    "p99_us": st.p99_us, "Guniforms_s": st.draws_completed / st.wall_s / 1e9})
        print(json.dumps(res), flush=True)
        return 0
    elif c.startswith("transform"):
        n = (1 << 30) // k
        d = srng.SRNG_DIST_NORMAL if c == "transform_normal" else srng.SRNG_DIST_EXPONENTIAL
        h = srng.srng_create(srng.SRNG_PHILOX4X32_10, 0xC0FFEE, 1, srng.SRNG_SPACING_STREAM, stream)
        u = torch.empty(n, dtype=torch.float32, device=dev)
        srng.srng_generate(h, 0, 1, n, srng.SRNG_OUT_F32, u, stream)
        o = torch.empty_like(u)
        fn = lambda: srng.srng_transform(d, u, n, o, stream)
        nbytes, nvals = n * 8, n
    else:
        gens, lengths, outoff = W.batched_instances(n_inst=W.BATCHED["n_inst"] // k)
        ni = len(gens)
        total = int(outoff[-1] + lengths[-1])
        h = srng.srng_create(srng.SRNG_MRG32K3A, SEED, ni, srng.SRNG_SPACING_STREAM, stream)
        h2 = srng.srng_create(srng.SRNG_PHILOX4X32_10, 0xC0FFEE, ni, srng.SRNG_SPACING_STREAM, stream)
        inst = [srng.Instance(set_index=int(gens[i]), stream=i, offset=0, length=int(lengths[i]),
                              out_offset=int(outoff[i])) for i in range(ni)]
        mode = srng.SRNG_BATCH_WRITE if c == "batch_write" else srng.SRNG_BATCH_FUSED_PI
        o = torch.empty(total if mode == 0 else ni, dtype=torch.int32 if mode == 0 else torch.int64, device=dev)
        plan = srng.srng_batch_plan_create([h, h2], inst, mode, srng.SRNG_OUT_U32, o, None, stream)
        fn = lambda: srng.srng_batch_plan_launch(plan, stream)
        nvals = int(sum(int(x) for x in lengths))
        nbytes = nvals * 4 if mode == 0 else ni * 8
    best, med = _time(torch, stream, fn, reps=args.reps, warm=1)
    res.update({"ms_best": best, "ms_median": med, "bytes": nbytes, "values": nvals,
                "GB_s": nbytes / best / 1e6, "Guniforms_s": nvals / best / 1e6})
    print(json.dumps(res), flush=True)
    return 0


CASES = {"mrg_u32", "mrg_f64", "mrg_plain", "philox_u32", "philox_f32", "philox_f64", "philox_normal", "philox_many_u32", "philox_keyed_many_u32",
         "threefry_u32", "threefry_f32", "threefry64_u32", "threefry64_f32",
         "tinymt_u32", "tinymt_f64",
         "batch_write", "batch_pi", "transform_exponential", "transform_normal", "serving"}


def main():
    args = parse()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
