"""CPU oracle for the bulk uniform-generation path (arXiv 1412.8266, ShoveRand).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this module.  It loads
``liboracle.so`` built from ``srng_oracle.c`` with plain gcc; it shares no code
with the CUDA library and never loads it.

The functions are thin numpy marshalling around the C definitions; each C
function states the passage of the paper it follows (MRG32k3a and sequence
splitting: Sec. 4.1 and Sec. 2.3; Philox4x32-10: Sec. 4.3) and the reading
taken where the paper is silent (seed expansion, conversions, the Monte Carlo
hit test, the Philox counter split).

Parity status per function (what pins it is in tests/test_oracle_pins.py):
  mrg_step / mrg_matpow / mrg_jump / mrg_stream_starts   pinned
  philox4x32_10 / philox_word                             pinned
  to_f32 / mrg_to_f64 / philox_to_f64                     pinned
  pi hit tests / pi counts                                pinned
  dist_constants / ln_unit_f32 / sincos_2pi_f32 / transform  pinned (exhaustive
      over the 2^24 FP32 uniforms against float64 libm, constants against
      exact rationals, distribution tests)
  threefry4x32_20 / threefry_word / threefry_*, and the
  threefry4x64_20 / threefry64_* counterparts              parity unpinned: the
      rotation counts and parity constant of Salmon et al. 2011 have no
      independent implementation here; structure pinned (bijection, key and
      counter use, the block-to-word layout, avalanche, and the round
      structure by an inverse written in tests/test_oracle_threefry.py that
      takes every block back to its counter)
  tinymt32_next / charpoly / max_period / jump / find_params  pinned (the
      authors' default parameter set has period 2^127 - 1 under the step,
      checked with sympy; the polynomial annihilates every state bit; jumps
      equal stepping and close the period)
  tinymt32_init                                            pinned: its mixing
      function is the MT19937 initialisation's, compared with numpy's MT19937
      seeding; the seeding rebuilt from that equals the oracle's
  tinymt32_temper                                          parity unpinned (the
      published TinyMT32 tempering restated; no implementation here to compare
      outputs with); structure pinned (the words it reads, the shift of s2,
      tmat exactly when the sum is odd, inverted to recover s3)
  splitmix64 / seed_expand (SplitMix64)                    pinned: every output
      equals pybind11's mix64 (the same finalizer, an independent
      implementation) of the Weyl sequence, whose step is the odd integer
      nearest 2^64/phi; the expanded state follows by mod m1 / m2
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srng_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

M1 = 4294967087
M2 = 4294944443
OUT_U32, OUT_F32, OUT_F64 = 0, 1, 2
_DTYPES = {OUT_U32: np.uint32, OUT_F32: np.float32, OUT_F64: np.float64}


def build(force: bool = False) -> str:
    """Compile srng_oracle.c into liboracle.so with gcc (no CUDA involved)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load(path: str | None = None):
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        if path is None:
            build()
        lib = ctypes.CDLL(path or _LIB_PATH)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        vp = ctypes.c_void_p
        u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        sig = {
            "oracle_mrg_step": (u32, [u32p]),
            "oracle_mrg_matrix": (None, [i32, u64p]),
            "oracle_mrg_matpow": (None, [i32, u64, u64, u64p]),
            "oracle_mrg_jump": (None, [u32p, u64, u64]),
            "oracle_mrg_stream_starts": (None, [u32p, i32, u64, u64, u32p]),
            "oracle_mrg_state_valid": (i32, [u32p]),
            "oracle_splitmix64_next": (u64, [u64p]),
            "oracle_seed_expand": (None, [u64, u32p]),
            "oracle_philox4x32_10": (None, [u32p, u32p, u32p]),
            "oracle_philox_word": (u32, [u32, u32, u64, u64]),
            "oracle_threefry4x32_20": (None, [u32p, u32p, u32p]),
            "oracle_threefry_word": (u32, [u64, u64, u64]),
            "oracle_threefry_generate": (None, [u64, u64, u64, u64, i32, vp]),
            "oracle_threefry_bulk": (None, [u64, u64, u64p, u64, u64, i32, vp, i32]),
            "oracle_threefry_pi_count": (ctypes.c_int64, [u64, u64, u64, u64]),
            "oracle_threefry4x64_20": (None, [u64p, u64p, u64p]),
            "oracle_threefry64_word": (u32, [u64, u64, u64]),
            "oracle_threefry64_generate": (None, [u64, u64, u64, u64, i32, vp]),
            "oracle_threefry64_pi_count": (ctypes.c_int64, [u64, u64, u64, u64]),
            "oracle_threefry64_bulk": (None, [u64, u64, u64p, u64, u64, i32, vp, i32]),
            "oracle_tinymt32_next": (None, [u32p, u32, u32]),
            "oracle_tinymt32_temper": (u32, [u32p, u32]),
            "oracle_tinymt32_init": (None, [u32, u32, u32, u32, u32p]),
            "oracle_tinymt32_charpoly": (i32, [u32, u32, ctypes.POINTER(ctypes.c_uint8)]),
            "oracle_tinymt32_max_period": (i32, [u32, u32]),
            "oracle_tinymt32_find_params": (None, [u64, u32, u32p]),
            "oracle_tinymt32_jump": (None, [u32p, u32, u32, u64, u64]),
            "oracle_tinymt32_stream_start": (None, [u32, u32p, u64, u32p]),
            "oracle_tinymt32_stream_starts": (None, [u32, u32p, u64, u64, u32p]),
            "oracle_tinymt32_generate": (None, [u32p, u32p, u64, i32, vp]),
            "oracle_tinymt32_bulk": (None, [u32p, u32p, u64, u64, u64, i32, vp, i32]),
            "oracle_to_f32": (ctypes.c_float, [u32]),
            "oracle_mrg_to_f64": (ctypes.c_double, [u32]),
            "oracle_dist_constants": (None, [ctypes.POINTER(ctypes.c_float)]),
            "oracle_ln_unit_f32": (ctypes.c_float, [ctypes.c_float]),
            "oracle_sincos_2pi_f32": (None, [ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                             ctypes.POINTER(ctypes.c_float)]),
            "oracle_transform": (None, [i32, vp, u64, vp]),
            "oracle_sincos_2pi_array": (None, [vp, u64, vp, vp]),
            "oracle_philox_to_f64": (ctypes.c_double, [u32]),
            "oracle_mrg_generate": (None, [u32p, u64, i32, vp]),
            "oracle_philox_generate": (None, [u32, u32, u64, u64, u64, i32, vp]),
            "oracle_mrg_bulk": (None, [u32p, u64, u64, i32, vp, i32]),
            "oracle_philox_bulk": (None, [u32, u32, u64, u64p, u64, u64, i32, vp, i32]),
            "oracle_pi_hit_philox": (i32, [u32, u32]),
            "oracle_pi_hit_mrg": (i32, [u32, u32]),
            "oracle_mrg_pi_count": (ctypes.c_int64, [u32p, u64]),
            "oracle_philox_pi_count": (ctypes.c_int64, [u32, u32, u64, u64, u64]),
            "oracle_batch": (None, [u64, vp, vp, u32, u32, vp, vp, vp, vp, i32, i32, vp, vp, i32]),
            "oracle_max_threads": (i32, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def use_library(path: str | None) -> None:
    """Test hook: route every oracle function through another build of
    srng_oracle.c (the mutation tests load deliberately broken copies);
    None returns to the regular build."""
    global _lib
    with _lock:
        _lib = None
    if path is not None:
        _load(path)


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _split128(n: int):
    if n < 0 or n >= 1 << 128:
        raise ValueError("jump distance must be in [0, 2^128)")
    return (n >> 64) & 0xFFFFFFFFFFFFFFFF, n & 0xFFFFFFFFFFFFFFFF


# ---------------------------------------------------------------- MRG32k3a
def mrg_step(state):
    """One step of MRG32k3a from a 6-word state; returns (z, new_state)."""
    s = np.array(state, dtype=np.uint32)
    z = _load().oracle_mrg_step(_u32p(s))
    return int(z), s


def mrg_matrix(comp: int) -> np.ndarray:
    a = np.zeros(9, dtype=np.uint64)
    _load().oracle_mrg_matrix(comp, _u64p(a))
    return a.reshape(3, 3)


def mrg_matpow(comp: int, e: int) -> np.ndarray:
    hi, lo = _split128(e)
    a = np.zeros(9, dtype=np.uint64)
    _load().oracle_mrg_matpow(comp, hi, lo, _u64p(a))
    return a.reshape(3, 3)


def mrg_jump(state, n: int) -> np.ndarray:
    s = np.array(state, dtype=np.uint32)
    hi, lo = _split128(n)
    _load().oracle_mrg_jump(_u32p(s), hi, lo)
    return s


def mrg_stream_starts(seed_state, e: int, first: int, count: int) -> np.ndarray:
    """Start states (count x 6) of streams first..first+count-1 spaced 2^e apart."""
    y0 = np.array(seed_state, dtype=np.uint32)
    out = np.zeros((count, 6), dtype=np.uint32)
    _load().oracle_mrg_stream_starts(_u32p(y0), e, first, count, _u32p(out))
    return out


def mrg_state_valid(state) -> bool:
    s = np.array(state, dtype=np.uint32)
    return bool(_load().oracle_mrg_state_valid(_u32p(s)))


def splitmix64(seed: int, n: int) -> list:
    st = (ctypes.c_uint64 * 1)(seed)
    lib = _load()
    p = ctypes.cast(st, ctypes.POINTER(ctypes.c_uint64))
    return [int(lib.oracle_splitmix64_next(p)) for _ in range(n)]


def seed_expand(seed: int) -> np.ndarray:
    out = np.zeros(6, dtype=np.uint32)
    _load().oracle_seed_expand(seed, _u32p(out))
    return out


def mrg_generate(state, n: int, out_type: int = OUT_U32):
    """n draws from a start state; returns (values, final_state)."""
    s = np.array(state, dtype=np.uint32)
    out = np.empty(n, dtype=_DTYPES[out_type])
    _load().oracle_mrg_generate(_u32p(s), n, out_type, out.ctypes.data_as(ctypes.c_void_p))
    return out, s


def mrg_bulk(states, n: int, out_type: int = OUT_U32, threads: int = 0):
    """Stream-major output (n_streams x n); states (n_streams x 6) advanced in place copy."""
    st = np.ascontiguousarray(np.array(states, dtype=np.uint32).reshape(-1, 6))
    out = np.empty((st.shape[0], n), dtype=_DTYPES[out_type])
    _load().oracle_mrg_bulk(_u32p(st), st.shape[0], n, out_type, out.ctypes.data_as(ctypes.c_void_p), threads)
    return out, st


# ---------------------------------------------------------------- Philox
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_u32p(c), _u32p(k), _u32p(out))
    return out


def philox_word(key, stream: int, pos: int) -> int:
    return int(_load().oracle_philox_word(key[0], key[1], stream, pos))


def philox_generate(key, stream: int, pos: int, n: int, out_type: int = OUT_U32) -> np.ndarray:
    out = np.empty(n, dtype=_DTYPES[out_type])
    _load().oracle_philox_generate(key[0], key[1], stream, pos, n, out_type, out.ctypes.data_as(ctypes.c_void_p))
    return out


def philox_keyed_generate(seed: int, stream: int, pos: int, n: int, out_type: int = OUT_U32) -> np.ndarray:
    """n words of stream `stream` in the keyed layout (reading of Sec. 4.3, the
    key set from the stream's own identifier): key = (stream low word, stream
    high word), counter words 2-3 = (seed low word, seed high word), counter
    words 0-1 = position / 4 -- the same Philox4x32-10 block with the roles of
    the key and counter words 2-3 exchanged."""
    return philox_generate((stream & 0xFFFFFFFF, stream >> 32), seed, pos, n, out_type)


def philox_bulk(key, stream0: int, positions, n: int, out_type: int = OUT_U32, threads: int = 0):
    pos = np.ascontiguousarray(np.array(positions, dtype=np.uint64))
    out = np.empty((pos.shape[0], n), dtype=_DTYPES[out_type])
    _load().oracle_philox_bulk(key[0], key[1], stream0, _u64p(pos), pos.shape[0], n, out_type,
                               out.ctypes.data_as(ctypes.c_void_p), threads)
    return out, pos


# ---------------------------------------------------------------- Threefry
def threefry4x32_20(ctr, key) -> np.ndarray:
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_threefry4x32_20(_u32p(c), _u32p(k), _u32p(out))
    return out


def threefry_word(seed: int, stream: int, pos: int) -> int:
    return int(_load().oracle_threefry_word(seed, stream, pos))


def threefry_generate(seed: int, stream: int, pos: int, n: int, out_type: int = OUT_U32) -> np.ndarray:
    out = np.empty(n, dtype=_DTYPES[out_type])
    _load().oracle_threefry_generate(seed, stream, pos, n, out_type, out.ctypes.data_as(ctypes.c_void_p))
    return out


def threefry_bulk(seed: int, stream0: int, positions, n: int, out_type: int = OUT_U32, threads: int = 0):
    pos = np.ascontiguousarray(np.array(positions, dtype=np.uint64))
    out = np.empty((pos.shape[0], n), dtype=_DTYPES[out_type])
    _load().oracle_threefry_bulk(seed, stream0, _u64p(pos), pos.shape[0], n, out_type,
                                 out.ctypes.data_as(ctypes.c_void_p), threads)
    return out, pos


def threefry_pi_count(seed: int, stream: int, pos: int, length: int) -> int:
    return int(_load().oracle_threefry_pi_count(seed, stream, pos, length))


def threefry4x64_20(ctr, key) -> np.ndarray:
    c = np.array(ctr, dtype=np.uint64)
    k = np.array(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().oracle_threefry4x64_20(_u64p(c), _u64p(k), _u64p(out))
    return out


def threefry64_word(seed: int, stream: int, pos: int) -> int:
    return int(_load().oracle_threefry64_word(seed, stream, pos))


def threefry64_generate(seed: int, stream: int, pos: int, n: int, out_type: int = OUT_U32) -> np.ndarray:
    out = np.empty(n, dtype=_DTYPES[out_type])
    _load().oracle_threefry64_generate(seed, stream, pos, n, out_type, out.ctypes.data_as(ctypes.c_void_p))
    return out


def threefry64_bulk(seed: int, stream0: int, positions, n: int, out_type: int = OUT_U32, threads: int = 0):
    pos = np.ascontiguousarray(np.array(positions, dtype=np.uint64))
    out = np.empty((pos.shape[0], n), dtype=_DTYPES[out_type])
    _load().oracle_threefry64_bulk(seed, stream0, _u64p(pos), pos.shape[0], n, out_type,
                                   out.ctypes.data_as(ctypes.c_void_p), threads)
    return out, pos


def threefry64_pi_count(seed: int, stream: int, pos: int, length: int) -> int:
    return int(_load().oracle_threefry64_pi_count(seed, stream, pos, length))


# ---------------------------------------------------------------- TinyMT32
def tinymt32_next(state, mat1: int, mat2: int) -> np.ndarray:
    s = np.array(state, dtype=np.uint32)
    _load().oracle_tinymt32_next(_u32p(s), mat1, mat2)
    return s


def tinymt32_temper(state, tmat: int) -> int:
    s = np.array(state, dtype=np.uint32)
    return int(_load().oracle_tinymt32_temper(_u32p(s), tmat))


def tinymt32_init(seed32: int, prm) -> np.ndarray:
    s = np.zeros(4, dtype=np.uint32)
    _load().oracle_tinymt32_init(seed32, prm[0], prm[1], prm[2], _u32p(s))
    return s


def tinymt32_charpoly(mat1: int, mat2: int) -> list:
    """Coefficients p[0..L] (p[i] of x^i) of the step's characteristic polynomial."""
    buf = (ctypes.c_uint8 * 256)()
    L = _load().oracle_tinymt32_charpoly(mat1, mat2, buf)
    return list(buf)[:L + 1]


def tinymt32_max_period(mat1: int, mat2: int) -> bool:
    return bool(_load().oracle_tinymt32_max_period(mat1, mat2))


def tinymt32_find_params(seed: int, count: int) -> np.ndarray:
    out = np.zeros((count, 3), dtype=np.uint32)
    _load().oracle_tinymt32_find_params(seed, count, _u32p(out))
    return out


def tinymt32_jump(state, mat1: int, mat2: int, J: int) -> np.ndarray:
    s = np.array(state, dtype=np.uint32)
    _load().oracle_tinymt32_jump(_u32p(s), mat1, mat2, (J >> 64) & (2**64 - 1), J & (2**64 - 1))
    return s


def tinymt32_stream_start(seed32: int, prm, j: int) -> np.ndarray:
    """Start state of stream j of a group: the seed state, then j * 2^64 steps."""
    p = np.ascontiguousarray(np.asarray(prm, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_tinymt32_stream_start(seed32, _u32p(p), j, _u32p(out))
    return out


def tinymt32_stream_starts(seed32: int, prm, group_size: int, n_streams: int) -> np.ndarray:
    """Start states (n_streams x 4): stream i uses parameter set i // group_size
    and starts (i mod group_size) 2^64 steps after that set's seed state."""
    prm = np.ascontiguousarray(np.asarray(prm, dtype=np.uint32).reshape(-1, 3))
    out = np.zeros((n_streams, 4), dtype=np.uint32)
    _load().oracle_tinymt32_stream_starts(seed32, _u32p(prm), group_size, n_streams, _u32p(out))
    return out


def tinymt32_generate(state, prm, n: int, out_type: int = OUT_U32):
    s = np.array(state, dtype=np.uint32)
    p = np.ascontiguousarray(np.asarray(prm, dtype=np.uint32))
    out = np.empty(n, dtype=_DTYPES[out_type])
    _load().oracle_tinymt32_generate(_u32p(s), _u32p(p), n, out_type, out.ctypes.data_as(ctypes.c_void_p))
    return out, s


def tinymt32_bulk(states, prm, group_size: int, n: int, out_type: int = OUT_U32, threads: int = 0):
    st = np.ascontiguousarray(np.array(states, dtype=np.uint32).reshape(-1, 4))
    p = np.ascontiguousarray(np.asarray(prm, dtype=np.uint32).reshape(-1, 3))
    out = np.empty((st.shape[0], n), dtype=_DTYPES[out_type])
    _load().oracle_tinymt32_bulk(_u32p(st), _u32p(p), group_size, st.shape[0], n, out_type,
                                 out.ctypes.data_as(ctypes.c_void_p), threads)
    return out, st


# ---------------------------------------------------------------- conversions
def to_f32(v: int) -> float:
    return float(_load().oracle_to_f32(v))


def mrg_to_f64(z: int) -> float:
    return float(_load().oracle_mrg_to_f64(z))


def philox_to_f64(w: int) -> float:
    return float(_load().oracle_philox_to_f64(w))


def convert(values: np.ndarray, gen: int, out_type: int) -> np.ndarray:
    """Vector form of the conversions, element by element through the C code."""
    lib = _load()
    v = np.asarray(values, dtype=np.uint32)
    if out_type == OUT_U32:
        return v.copy()
    if out_type == OUT_F32:
        return np.array([lib.oracle_to_f32(int(x)) for x in v], dtype=np.float32)
    f = lib.oracle_mrg_to_f64 if gen == 0 else lib.oracle_philox_to_f64
    return np.array([f(int(x)) for x in v], dtype=np.float64)


# ---------------------------------------------------------------- Monte Carlo pi
def pi_hit_philox(w0: int, w1: int) -> bool:
    return bool(_load().oracle_pi_hit_philox(w0, w1))


def pi_hit_mrg(z0: int, z1: int) -> bool:
    return bool(_load().oracle_pi_hit_mrg(z0, z1))


def mrg_pi_count(state, length: int) -> int:
    s = np.array(state, dtype=np.uint32)
    return int(_load().oracle_mrg_pi_count(_u32p(s), length))


def philox_pi_count(key, stream: int, pos: int, length: int) -> int:
    return int(_load().oracle_philox_pi_count(key[0], key[1], stream, pos, length))


# ---------------------------------------------------------------- batches
def batch(gens, mrg_states, key, philox_streams, philox_pos, lengths, out_offsets, mode: int,
          out_type: int = OUT_U32, total: int | None = None, threads: int = 0):
    """Batched instances (see oracle_batch in srng_oracle.c).  Returns the flat
    output array (mode 0) or the int64 hit counts (mode 1)."""
    g = np.ascontiguousarray(np.asarray(gens, dtype=np.int32))
    n = g.shape[0]
    ms = np.ascontiguousarray(np.asarray(mrg_states, dtype=np.uint32).reshape(n, 6))
    ps = np.ascontiguousarray(np.asarray(philox_streams, dtype=np.uint64))
    pp = np.ascontiguousarray(np.asarray(philox_pos, dtype=np.uint64))
    ln = np.ascontiguousarray(np.asarray(lengths, dtype=np.uint64))
    oo = np.ascontiguousarray(np.asarray(out_offsets, dtype=np.uint64))
    counts = np.zeros(n, dtype=np.int64)
    if mode == 0:
        if total is None:
            total = int((oo + ln).max()) if n else 0
        out = np.zeros(total, dtype=_DTYPES[out_type])
        outp = out.ctypes.data_as(ctypes.c_void_p)
    else:
        out = None
        outp = None
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _load().oracle_batch(n, vp(g), vp(ms), key[0], key[1], vp(ps), vp(pp), vp(ln), vp(oo), mode,
                         out_type, outp, vp(counts), threads)
    return out if mode == 0 else counts


DIST_EXPONENTIAL, DIST_NORMAL = 0, 1


def dist_constants() -> dict:
    """The single-precision constants the variate transforms use."""
    buf = (ctypes.c_float * 18)()
    _load().oracle_dist_constants(buf)
    v = list(buf)
    return {"ln2_hi": v[0], "ln2_lo": v[1], "inv_odd": v[2:8], "sc": [None] + v[8:18]}


def ln_unit_f32(x: float) -> float:
    return float(_load().oracle_ln_unit_f32(x))


def sincos_2pi_f32(u: float):
    s, c = ctypes.c_float(), ctypes.c_float()
    _load().oracle_sincos_2pi_f32(u, ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def sincos_2pi_array(u: np.ndarray):
    u = np.ascontiguousarray(u, dtype=np.float32)
    s, c = np.empty_like(u), np.empty_like(u)
    _load().oracle_sincos_2pi_array(u.ctypes.data, u.size, s.ctypes.data, c.ctypes.data)
    return s, c


def transform(dist: int, u: np.ndarray) -> np.ndarray:
    """Exponential (dist 0) or Box-Muller normal (dist 1, even length)
    variates from FP32 uniforms in [0, 1)."""
    u = np.ascontiguousarray(u, dtype=np.float32)
    if dist == DIST_NORMAL and u.size % 2:
        raise ValueError("normal variates come in pairs")
    out = np.empty_like(u)
    _load().oracle_transform(dist, u.ctypes.data, u.size, out.ctypes.data)
    return out


def max_threads() -> int:
    return int(_load().oracle_max_threads())
