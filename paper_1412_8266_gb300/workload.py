"""Seeded synthetic workloads (inputs only: no generator arithmetic here).

Both the CUDA path and the CPU oracle receive the lists built here; neither
side draws its inputs itself.  The random draws use numpy's PCG64
(``numpy.random.default_rng``) with fixed seeds, a generator unrelated to the
generators under test.

Workloads (sizes as in the configurations this library is measured on):
  mrg_plain    MRG32k3a, seed state all 12345, 64 streams 2^127 apart,
               2^16 FP64 draws per stream.
  mrg_bulk     MRG32k3a, seed 0x5EED5EED5EED5EED expanded to six words,
               2^18 streams x 4096 draws, as uint32 and as FP64.
  philox_bulk  Philox4x32-10, key from seed 0xC0FFEE, counters 0 .. 2^28-1
               (one stream, 2^30 words), as uint32 and as FP32.
  batched      10,000 instances, lengths log-uniform in [1e2, 1e7], even
               instances MRG32k3a (stream i of a mrg_bulk-seeded set), odd
               instances Philox (stream i under the philox_bulk key); output
               slots at prefix-sum offsets rounded up to 32 bytes.
  serving      Poisson arrivals at 20,000 requests/s, n log-uniform in
               [1e3, 1e8] FP32 draws, stream uniform over 10^6 MRG32k3a
               substreams of the all-12345 state; 16 GB output budget.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MRG_PLAIN = dict(name="MRG32k3a plain: 64 streams spaced 2^127, 2^16 FP64 each (all-12345 seed state)",
                 seed_state=[12345] * 6, n_streams=64, n=1 << 16)
MRG_BULK = dict(name="MRG32k3a bulk: 2^18 streams x 4096 draws, uint32 + FP64",
                seed=0x5EED5EED5EED5EED, n_streams=1 << 18, n=4096)
PHILOX_BULK = dict(name="Philox4x32-10 bulk: key 0xC0FFEE, counters 0..2^28-1 (2^30 words), uint32 + FP32",
                   seed=0xC0FFEE, n_streams=1, n=1 << 30)
BATCHED = dict(name="Batched uneven: 10^4 instances, lengths log-uniform [1e2, 1e7], half MRG32k3a / half Philox",
               n_inst=10_000, lo=1e2, hi=1e7, length_seed=20141226)
SERVING = dict(name="Serving: Poisson 20k req/s, n log-uniform [1e3, 1e8] FP32, 1e6 MRG32k3a substreams, 16 GB budget",
               rate=20_000.0, lo=1e3, hi=1e8, n_streams=1_000_000, budget=16 << 30, trace_seed=1412_8266)


def log_uniform_ints(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """n integers floor(exp(ln lo + u ln(hi/lo))), u uniform in [0, 1)."""
    u = np.random.default_rng(seed).random(n)
    a, b = math.log(lo), math.log(hi / lo)
    return np.array([int(math.floor(math.exp(a + x * b))) for x in u], dtype=np.uint64)


def batched_instances(n_inst: int = BATCHED["n_inst"], lo: float = BATCHED["lo"], hi: float = BATCHED["hi"],
                      seed: int = BATCHED["length_seed"], align: int = 8):
    """Returns (gens, lengths, out_offsets): gens[i] = 0 (MRG32k3a) for even i,
    1 (Philox) for odd i; instance i's output slot starts at the prefix sum of
    the earlier lengths, each slot rounded up to a multiple of `align`
    elements (8 x 4 bytes: every slot starts on a 32-byte boundary; align=1
    packs the slots back to back)."""
    lengths = log_uniform_ints(n_inst, lo, hi, seed)
    gens = np.array([i % 2 for i in range(n_inst)], dtype=np.int32)
    slots = (lengths + np.uint64(align - 1)) // np.uint64(align) * np.uint64(align)
    offs = np.zeros(n_inst, dtype=np.uint64)
    if n_inst > 1:
        offs[1:] = np.cumsum(slots[:-1], dtype=np.uint64)
    return gens, lengths, offs


@dataclass
class Request:
    arrival_s: float
    stream: int
    n: int


def serving_trace(duration_s: float, rate: float = SERVING["rate"], lo: float = SERVING["lo"],
                  hi: float = SERVING["hi"], n_streams: int = SERVING["n_streams"],
                  seed: int = SERVING["trace_seed"]) -> list:
    """Poisson arrivals (exponential gaps of mean 1/rate) over duration_s."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    a, b = math.log(lo), math.log(hi / lo)
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration_s:
            break
        n = int(math.floor(math.exp(a + float(rng.random()) * b)))
        s = int(rng.integers(0, n_streams))
        out.append(Request(t, s, n))
    return out
