"""Launch-shape autotuner for the generation and batch kernels.

Outputs never depend on the launch shape (tested); only speed does.  The
tuner times every candidate of a small search space through the C ABI
(``srng_generate_tuned`` / a batch plan per candidate) with CUDA events on the
launching stream, keeps the fastest, installs it with ``srng_set_tune`` and
records it in a JSON cache keyed by generator, output type, problem-size class
and device (name and SM count).

Search spaces (all values valid for every problem):
  MRG32k3a  block_threads x resident blocks/SM x chunk (draws per thread item)
            x store path (shared-memory staged rows or direct per-lane rows;
            for FP64 also direct rows with three in eight doubles through
            the FP64 multiply) x resident blocks per SM for the direct rows
  Philox    block_threads x unroll (blocks per thread per trip) x blocks/SM
  batch     chunk (MRG32k3a) x lane_blocks (Philox) per work item
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time

import paper_1412_8266_gb300 as srng

MRG_SPACE = [dict(block_threads=bt, blocks_per_sm=b, chunk=c, vector_store=v)
             for bt, b, c, v in itertools.product((128, 256), (4, 8), (512, 1024, 2048, 4096), (1, 3))]
# 4-byte values add the direct rows held to 6 resident blocks per SM (2^18 x 4096
# uint32 in items of 2048: 1.150 ms, against 1.229 with no limit), also with
# grids of 16 and 32 blocks per SM: more blocks than fit at once, which the
# block scheduler hands out as others finish, so no SM waits through a partial
# last grid-stride pass (items of 1024: 1.107 ms, against 1.173 with 8)
MRG_SPACE_4B = MRG_SPACE + [dict(block_threads=bt, blocks_per_sm=b, chunk=c, vector_store=3, resident=6)
                            for bt, b, c in itertools.product((128, 256), (4, 8, 16, 32), (512, 1024, 2048, 4096))]
# FP64 adds the direct rows with three in eight doubles through the FP64 multiply
# (with at most 6 resident blocks per SM, the FP64 default, or as many as fit:
# 32), on grids of 4 to 32 blocks per SM (items of 1024, 16 per SM: 1.621 ms,
# against 1.686 for the best with 8)
MRG_SPACE_F64 = MRG_SPACE + [dict(block_threads=bt, blocks_per_sm=b, chunk=c, vector_store=4, resident=r)
                             for bt, b, c, r in itertools.product((128, 256), (4, 8, 16, 32),
                                                                  (512, 1024, 2048, 4096), (6, 32))]
PHILOX_SPACE = [dict(block_threads=bt, unroll=u, blocks_per_sm=b)
                for bt, u, b in itertools.product((128, 256), (1, 2, 4), (4, 8, 16, 32))]
BATCH_SPACE = [dict(chunk=c, lane_blocks=lb) for c, lb in itertools.product((256, 512, 1024, 2048, 4096),
                                                                              (32, 64, 128, 256))]


def cache_path() -> str:
    return os.environ.get("SRNG_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "srng_gb300",
                                                           "tune.json"))


def _device_key(torch):
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}/{p.multi_processor_count}sm"


def size_class(n_values: int) -> str:
    return f"2^{int(math.log2(max(1, n_values)))}"


def _load_cache():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _save_cache(d):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _time_ms(torch, stream, fn, reps):
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_generate(gen: int, out_type: int, n_streams: int, n_per_stream: int, space=None, reps: int = 3,
                  use_cache: bool = True, install: bool = True, seed: int = 0x5EED5EED5EED5EED):
    """Pick the fastest launch shape for srng_generate of (gen, out_type) on a
    problem of n_streams x n_per_stream; returns (best tune dict, {repr: ms})."""
    import torch
    key = f"generate/{gen}/{out_type}/{size_class(n_streams)}x{size_class(n_per_stream)}/{_device_key(torch)}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        best = cache[key]["tune"]
        if install:
            srng.srng_set_tune(gen, out_type, best)
        return best, cache[key].get("table", {})
    if not space:
        if gen == srng.SRNG_MRG32K3A:
            space = MRG_SPACE_F64 if out_type == srng.SRNG_OUT_F64 else MRG_SPACE_4B
        else:
            space = PHILOX_SPACE
    stream = torch.cuda.current_stream()
    h = srng.srng_create(gen, seed, n_streams, srng.SRNG_SPACING_STREAM, stream)
    item = 8 if out_type == srng.SRNG_OUT_F64 else 4
    out = torch.empty(n_streams * n_per_stream * item, dtype=torch.uint8, device="cuda")
    table = {}
    try:
        for cand in space:
            def fn(c=cand):
                srng.srng_reset(h, stream)
                srng.srng_generate_tuned(h, 0, n_streams, n_per_stream, out_type, out, c, stream)
            table[json.dumps(cand, sort_keys=True)] = _time_ms(torch, stream, fn, reps)
    finally:
        srng.srng_destroy(h)
        del out
    best = json.loads(min(table, key=table.get))
    if install:
        srng.srng_set_tune(gen, out_type, best)
    if use_cache:
        cache = _load_cache()
        cache[key] = {"tune": best, "table": table, "when": time.time()}
        _save_cache(cache)
    return best, table


def tune_batch(sets, inst, mode: int, out_type: int, out, space=None, reps: int = 3):
    """Pick chunk / lane_blocks for a batch; returns (best tune dict, {repr: ms})."""
    import torch
    stream = torch.cuda.current_stream()
    table = {}
    for cand in (space or BATCH_SPACE):
        plan = srng.srng_batch_plan_create(sets, inst, mode, out_type, out, cand, stream)
        try:
            table[json.dumps(cand, sort_keys=True)] = _time_ms(torch, stream,
                                                               lambda: srng.srng_batch_plan_launch(plan, stream), reps)
        finally:
            srng.srng_batch_plan_destroy(plan)
    best = json.loads(min(table, key=table.get))
    return best, table
