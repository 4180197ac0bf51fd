"""Python binding of the GB300 bulk uniform-generation library (include/srng.h).

Argument marshalling only: every function here has the name of the C entry
point it calls, passes plain pointers and sizes through ``ctypes``, and raises
``SrngError`` when the call returns a non-zero status.  All generation runs in
the CUDA kernels of ``libsrng.so``; there is no fallback of any kind -- if the
library is missing or cannot be loaded, every call raises.

Pointers may be given as integers, ``torch.Tensor`` (its ``data_ptr()``) or
numpy arrays (host pointers).  ``stream`` may be ``None`` (torch's current
stream when torch is imported and CUDA is initialised, else the legacy
default stream), an integer ``cudaStream_t`` or a ``torch.cuda.Stream``.
"""
from __future__ import annotations

import ctypes
import os
import sys
import threading

__all__ = [
    "SrngError", "Tune", "Instance", "SetDesc", "DevView", "ServerConfig", "ServerStats", "Request",
    "lib_path", "load",
    "SRNG_MRG32K3A", "SRNG_PHILOX4X32_10", "SRNG_PHILOX4X32_10_KEYED", "SRNG_THREEFRY4X32_20", "SRNG_THREEFRY4X64_20", "SRNG_TINYMT32",
    "SRNG_OUT_U32", "SRNG_OUT_F32", "SRNG_OUT_F64", "SRNG_OUT_EXP_F32", "SRNG_OUT_NORMAL_F32",
    "SRNG_SPACING_STREAM", "SRNG_SPACING_SUBSTREAM", "SRNG_JUMP_DRAWS", "SRNG_JUMP_SUBSTREAMS",
    "SRNG_JUMP_STREAMS", "SRNG_BATCH_WRITE", "SRNG_BATCH_FUSED_PI", "SRNG_DIST_EXPONENTIAL", "SRNG_DIST_NORMAL",
]

SRNG_ABI_VERSION = 3  # the struct layouts below follow this version of include/srng.h
SRNG_MRG32K3A, SRNG_PHILOX4X32_10, SRNG_PHILOX4X32_10_KEYED, SRNG_THREEFRY4X32_20, SRNG_TINYMT32 = 0, 1, 2, 3, 4
SRNG_THREEFRY4X64_20 = 5
SRNG_OUT_U32, SRNG_OUT_F32, SRNG_OUT_F64 = 0, 1, 2
SRNG_OUT_EXP_F32, SRNG_OUT_NORMAL_F32 = 3, 4
SRNG_SPACING_STREAM, SRNG_SPACING_SUBSTREAM = 0, 1
SRNG_JUMP_DRAWS, SRNG_JUMP_SUBSTREAMS, SRNG_JUMP_STREAMS = 0, 1, 2
SRNG_BATCH_WRITE, SRNG_BATCH_FUSED_PI = 0, 1
SRNG_DIST_EXPONENTIAL, SRNG_DIST_NORMAL = 0, 1
OUT_ITEMSIZE = {SRNG_OUT_U32: 4, SRNG_OUT_F32: 4, SRNG_OUT_F64: 8}

STATUS_NAMES = {0: "SRNG_OK", 1: "SRNG_ERR_ARG", 2: "SRNG_ERR_OOM", 3: "SRNG_ERR_STATE", 4: "SRNG_ERR_CUDA",
                5: "SRNG_ERR_BUDGET", 6: "SRNG_ERR_TIMEOUT", 7: "SRNG_ERR_RANGE", 8: "SRNG_ERR_CLOSED",
                9: "SRNG_ERR_UNSUPPORTED"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None


class SrngError(RuntimeError):
    def __init__(self, status: int, message: str, func: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{func}: {self.name}: {message}")


class Tune(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("chunk", ctypes.c_uint32), ("unroll", ctypes.c_uint32), ("vector_store", ctypes.c_uint32),
                ("lane_blocks", ctypes.c_uint32), ("resident", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class Instance(ctypes.Structure):
    _fields_ = [("set_index", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("stream", ctypes.c_uint64),
                ("offset", ctypes.c_uint64), ("length", ctypes.c_uint64), ("out_offset", ctypes.c_uint64)]


class SetDesc(ctypes.Structure):
    _fields_ = [("gen", ctypes.c_int), ("spacing", ctypes.c_int), ("n_streams", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("seed_state", ctypes.c_uint32 * 6), ("stream_base", ctypes.c_uint64)]


class DevView(ctypes.Structure):
    _fields_ = [("gen", ctypes.c_int32), ("key0", ctypes.c_uint32), ("key1", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("n_streams", ctypes.c_uint64), ("mrg_state", ctypes.c_void_p),
                ("philox_pos", ctypes.c_void_p), ("stream_base", ctypes.c_uint64),
                ("tinymt_state", ctypes.c_void_p), ("tinymt_params", ctypes.c_void_p),
                ("tinymt_group_size", ctypes.c_uint64)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("max_step_requests", ctypes.c_uint32), ("max_step_draws", ctypes.c_uint64),
                ("chunk", ctypes.c_uint32), ("lane_blocks", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 4)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("draws_completed", ctypes.c_uint64), ("steps", ctypes.c_uint64), ("kernels", ctypes.c_uint64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("wall_s", ctypes.c_double), ("peak_pool_bytes", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("stream", ctypes.c_uint64), ("n", ctypes.c_uint64)]


_vp, _u64, _u32, _int = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
_SIGS = {
    "srng_last_error": (ctypes.c_char_p, []),
    "srng_status_string": (ctypes.c_char_p, [_int]),
    "srng_abi_version": (_int, []),
    "srng_create": (_int, [ctypes.POINTER(_vp), _int, _u64, _u64, _int, _vp]),
    "srng_create_from_state": (_int, [ctypes.POINTER(_vp), _vp, _u64, _int, _vp]),
    "srng_create_range": (_int, [ctypes.POINTER(_vp), _int, _u64, _vp, _u64, _u64, _int, _vp]),
    "srng_create_tinymt": (_int, [ctypes.POINTER(_vp), _vp, _u64, _u64, _u64, _vp]),
    "srng_tinymt_find_params": (_int, [_u64, _u32, _vp]),
    "srng_tinymt_check_params": (_int, [_u32, _u32, ctypes.POINTER(_int)]),
    "srng_destroy": (_int, [_vp]),
    "srng_reset": (_int, [_vp, _vp]),
    "srng_describe": (_int, [_vp, ctypes.POINTER(SetDesc)]),
    "srng_get_device_view": (_int, [_vp, ctypes.POINTER(DevView)]),
    "srng_jump": (_int, [_vp, _u64, _u64, _int, _u64, _u64, _vp]),
    "srng_generate": (_int, [_vp, _u64, _u64, _u64, _int, _vp, _vp]),
    "srng_generate_tuned": (_int, [_vp, _u64, _u64, _u64, _int, _vp, ctypes.POINTER(Tune), _vp]),
    "srng_generate_host": (_int, [_vp, _u64, _u64, _u64, _int, _vp, _vp]),
    "srng_get_state": (_int, [_vp, _u64, _u64, _vp, _vp]),
    "srng_set_state": (_int, [_vp, _u64, _u64, _vp, _vp]),
    "srng_set_tune": (_int, [_int, _int, ctypes.POINTER(Tune)]),
    "srng_get_tune": (_int, [_int, _int, ctypes.POINTER(Tune)]),
    "srng_convert": (_int, [_int, _int, _vp, _u64, _vp, _vp]),
    "srng_transform": (_int, [_int, _vp, _u64, _vp, _vp]),
    "srng_seed_expand": (_int, [_u64, _vp]),
    "srng_jump_matrix": (_int, [_int, _u64, _u64, _vp, _vp]),
    "srng_batch_plan_create": (_int, [ctypes.POINTER(_vp), _vp, _u32, _vp, _u64, _int, _int, _vp,
                                      ctypes.POINTER(Tune), _vp]),
    "srng_batch_plan_launch": (_int, [_vp, _vp]),
    "srng_batch_plan_info": (_int, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u32)]),
    "srng_batch_plan_destroy": (_int, [_vp]),
    "srng_batch_run": (_int, [_vp, _u32, _vp, _u64, _int, _int, _vp, _vp]),
    "srng_batch_run_static": (_int, [_vp, _u32, _vp, _u64, _int, _int, _vp, _vp]),
    "srng_server_create": (_int, [ctypes.POINTER(_vp), _vp, ctypes.POINTER(ServerConfig)]),
    "srng_server_submit": (_int, [_vp, _u64, _u64, _int, ctypes.POINTER(_u64)]),
    "srng_server_submit_at": (_int, [_vp, _u64, _u64, _u64, _int, ctypes.POINTER(_u64)]),
    "srng_server_poll": (_int, [_vp, _u64, ctypes.POINTER(_int), ctypes.POINTER(_vp)]),
    "srng_server_wait": (_int, [_vp, _u64, _u32, ctypes.POINTER(_vp)]),
    "srng_server_release": (_int, [_vp, _u64]),
    "srng_server_read": (_int, [_vp, _u64, _vp, _int]),
    "srng_server_get_stats": (_int, [_vp, ctypes.POINTER(ServerStats)]),
    "srng_server_reset_stats": (_int, [_vp]),
    "srng_server_destroy": (_int, [_vp]),
    "srng_server_replay": (_int, [_vp, _vp, _u64, _int, ctypes.c_double, _u32, ctypes.POINTER(ServerStats)]),
}


def lib_path() -> str:
    return os.path.join(_HERE, "libsrng.so")


def load():
    """Load libsrng.so (built by ``__graft_entry__.build()``).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libsrng.so not found at {path}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(st: int, func: str):
    if st != 0:
        msg = load().srng_last_error()
        raise SrngError(st, msg.decode() if msg else "", func)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    if isinstance(x, ctypes.Array):
        return ctypes.addressof(x)
    raise TypeError(f"cannot take a pointer of {type(x)!r}")


def _out_size(out_type: int) -> int:
    return 8 if out_type == SRNG_OUT_F64 else 4


def _buffer(x, nbytes: int, func: str, where: str = "any") -> int:
    """Pointer of a caller-owned buffer after checking what the binding can see:
    a torch tensor or numpy array must be contiguous, large enough for the
    nbytes the call writes or reads, and on the side the call expects
    ("cuda", "host" or "any").  Raw integer addresses pass unchecked."""
    if x is None or isinstance(x, int):
        return _ptr(x)
    size = None
    if hasattr(x, "data_ptr") and hasattr(x, "element_size"):  # torch
        if not x.is_contiguous():
            raise ValueError(f"{func}: the buffer must be contiguous")
        if where == "cuda" and not x.is_cuda:
            raise ValueError(f"{func}: expects a CUDA buffer, got one on {x.device}")
        if where == "host" and x.is_cuda:
            raise ValueError(f"{func}: expects a host buffer, got one on {x.device}")
        size = x.numel() * x.element_size()
    elif hasattr(x, "ctypes") and hasattr(x, "nbytes"):  # numpy
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{func}: the buffer must be contiguous")
        if where == "cuda":
            raise ValueError(f"{func}: expects a CUDA buffer, got a host array")
        size = x.nbytes
    elif isinstance(x, ctypes.Array):
        size = ctypes.sizeof(x)
    if size is not None and size < nbytes:
        raise ValueError(f"{func}: the buffer holds {size} bytes, the call needs {nbytes}")
    return _ptr(x)


def _stream(s) -> int:
    if s is None:
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
            return int(torch.cuda.current_stream().cuda_stream)
        return 0
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    raise TypeError(f"not a stream: {type(s)!r}")


def _tune(t):
    if t is None:
        return None
    if isinstance(t, Tune):
        return ctypes.byref(t)
    if isinstance(t, dict):
        return ctypes.byref(Tune(**t))
    raise TypeError("tune must be a Tune or a dict")


# ---------------------------------------------------------------- errors / info
def srng_last_error() -> str:
    return load().srng_last_error().decode()


def srng_status_string(status: int) -> str:
    return load().srng_status_string(status).decode()


def srng_abi_version() -> int:
    return load().srng_abi_version()


# ---------------------------------------------------------------- stream sets
def srng_create(gen: int, seed: int, n_streams: int, spacing: int = SRNG_SPACING_STREAM, stream=None) -> int:
    h = _vp()
    _check(load().srng_create(ctypes.byref(h), gen, seed, n_streams, spacing, _stream(stream)), "srng_create")
    return h.value


def srng_create_tinymt(params, group_size: int, seed: int, stream=None) -> int:
    """params: (mat1, mat2, tmat) per parameter set (n x 3); each set serves
    group_size consecutive streams."""
    import numpy as np
    p = np.ascontiguousarray(np.asarray(params, dtype=np.uint32).reshape(-1, 3))
    h = _vp()
    _check(load().srng_create_tinymt(ctypes.byref(h), p.ctypes.data, p.shape[0], group_size, seed, _stream(stream)),
           "srng_create_tinymt")
    return h.value


def srng_tinymt_find_params(seed: int, count: int):
    import numpy as np
    out = np.zeros((count, 3), dtype=np.uint32)
    _check(load().srng_tinymt_find_params(seed, count, out.ctypes.data), "srng_tinymt_find_params")
    return out


def srng_tinymt_check_params(mat1: int, mat2: int) -> bool:
    ok = _int()
    _check(load().srng_tinymt_check_params(mat1, mat2, ctypes.byref(ok)), "srng_tinymt_check_params")
    return bool(ok.value)


def srng_create_from_state(state, n_streams: int, spacing: int = SRNG_SPACING_STREAM, stream=None) -> int:
    st = (ctypes.c_uint32 * 6)(*[int(x) for x in state])
    h = _vp()
    _check(load().srng_create_from_state(ctypes.byref(h), ctypes.addressof(st), n_streams, spacing,
                                         _stream(stream)), "srng_create_from_state")
    return h.value


def srng_create_range(gen: int, seed: int, stream_base: int, n_streams: int, spacing: int = SRNG_SPACING_STREAM,
                      state=None, stream=None) -> int:
    st = None if state is None else (ctypes.c_uint32 * 6)(*[int(x) for x in state])
    h = _vp()
    _check(load().srng_create_range(ctypes.byref(h), gen, seed, ctypes.addressof(st) if st is not None else None,
                                    stream_base, n_streams, spacing, _stream(stream)), "srng_create_range")
    return h.value


def srng_destroy(handle: int) -> None:
    _check(load().srng_destroy(handle), "srng_destroy")


def srng_reset(handle: int, stream=None) -> None:
    _check(load().srng_reset(handle, _stream(stream)), "srng_reset")


def srng_describe(handle: int) -> SetDesc:
    d = SetDesc()
    _check(load().srng_describe(handle, ctypes.byref(d)), "srng_describe")
    return d


def srng_get_device_view(handle: int) -> DevView:
    v = DevView()
    _check(load().srng_get_device_view(handle, ctypes.byref(v)), "srng_get_device_view")
    return v


def srng_jump(handle: int, stream_begin: int, count: int, unit: int, n: int, stream=None) -> None:
    _check(load().srng_jump(handle, stream_begin, count, unit, (n >> 64) & (2**64 - 1), n & (2**64 - 1),
                            _stream(stream)), "srng_jump")


def srng_generate(handle: int, stream_begin: int, stream_count: int, n_per_stream: int, out_type: int, out,
                  stream=None) -> None:
    p = _buffer(out, stream_count * n_per_stream * _out_size(out_type), "srng_generate", "cuda")
    _check(load().srng_generate(handle, stream_begin, stream_count, n_per_stream, out_type, p, _stream(stream)),
           "srng_generate")


def srng_generate_tuned(handle: int, stream_begin: int, stream_count: int, n_per_stream: int, out_type: int, out,
                        tune=None, stream=None) -> None:
    p = _buffer(out, stream_count * n_per_stream * _out_size(out_type), "srng_generate_tuned", "cuda")
    _check(load().srng_generate_tuned(handle, stream_begin, stream_count, n_per_stream, out_type, p,
                                      _tune(tune), _stream(stream)), "srng_generate_tuned")


def srng_generate_host(handle: int, stream_begin: int, stream_count: int, n_per_stream: int, out_type: int,
                       out_host, stream=None) -> None:
    p = _buffer(out_host, stream_count * n_per_stream * _out_size(out_type), "srng_generate_host", "host")
    _check(load().srng_generate_host(handle, stream_begin, stream_count, n_per_stream, out_type, p,
                                     _stream(stream)), "srng_generate_host")


def _state_bytes(handle: int) -> int:
    """Bytes of host state per stream (srng_get_state / srng_set_state)."""
    gen = srng_describe(handle).gen
    return 24 if gen == SRNG_MRG32K3A else 16 if gen == SRNG_TINYMT32 else 8


def srng_get_state(handle: int, stream_begin: int, count: int, state_host, stream=None) -> None:
    p = _buffer(state_host, count * _state_bytes(handle), "srng_get_state", "host")
    _check(load().srng_get_state(handle, stream_begin, count, p, _stream(stream)), "srng_get_state")


def srng_set_state(handle: int, stream_begin: int, count: int, state_host, stream=None) -> None:
    p = _buffer(state_host, count * _state_bytes(handle), "srng_set_state", "host")
    _check(load().srng_set_state(handle, stream_begin, count, p, _stream(stream)), "srng_set_state")


def srng_set_tune(gen: int, out_type: int, tune=None) -> None:
    _check(load().srng_set_tune(gen, out_type, _tune(tune)), "srng_set_tune")


def srng_get_tune(gen: int, out_type: int) -> Tune:
    t = Tune()
    _check(load().srng_get_tune(gen, out_type, ctypes.byref(t)), "srng_get_tune")
    return t


def srng_convert(gen: int, out_type: int, in_dev, n: int, out_dev, stream=None) -> None:
    pi = _buffer(in_dev, 4 * n, "srng_convert", "cuda")
    po = _buffer(out_dev, n * _out_size(out_type), "srng_convert", "cuda")
    _check(load().srng_convert(gen, out_type, pi, n, po, _stream(stream)), "srng_convert")


def srng_transform(dist: int, in_dev, n: int, out_dev, stream=None) -> None:
    pi = _buffer(in_dev, 4 * n, "srng_transform", "cuda")
    po = _buffer(out_dev, 4 * n, "srng_transform", "cuda")
    _check(load().srng_transform(dist, pi, n, po, _stream(stream)), "srng_transform")


def srng_seed_expand(seed: int) -> list:
    st = (ctypes.c_uint32 * 6)()
    _check(load().srng_seed_expand(seed, ctypes.addressof(st)), "srng_seed_expand")
    return list(st)


def srng_jump_matrix(unit: int, n: int):
    a1 = (ctypes.c_uint32 * 9)()
    a2 = (ctypes.c_uint32 * 9)()
    _check(load().srng_jump_matrix(unit, (n >> 64) & (2**64 - 1), n & (2**64 - 1), ctypes.addressof(a1),
                                   ctypes.addressof(a2)), "srng_jump_matrix")
    return [list(a1[3 * i:3 * i + 3]) for i in range(3)], [list(a2[3 * i:3 * i + 3]) for i in range(3)]


# ---------------------------------------------------------------- batches
def _instances(inst):
    if isinstance(inst, ctypes.Array):
        return inst, len(inst)
    arr = (Instance * len(inst))()
    for i, x in enumerate(inst):
        if isinstance(x, Instance):
            arr[i] = x
        else:
            arr[i] = Instance(**x) if isinstance(x, dict) else Instance(*x)
    return arr, len(inst)


def _sets(sets):
    arr = (_vp * len(sets))(*sets)
    return arr, len(sets)


def _batch_out_bytes(ia, ni: int, mode: int, out_type: int) -> int:
    if mode == SRNG_BATCH_FUSED_PI:
        return 8 * ni
    return max((ia[i].out_offset + ia[i].length for i in range(ni)), default=0) * _out_size(out_type)


def srng_batch_plan_create(sets, inst, mode: int, out_type: int, out_dev, tune=None, stream=None):
    """Returns the plan handle; the plan keeps out_dev's address."""
    sa, ns = _sets(sets)
    ia, ni = _instances(inst)
    p = _buffer(out_dev, _batch_out_bytes(ia, ni, mode, out_type), "srng_batch_plan_create", "cuda")
    h = _vp()
    _check(load().srng_batch_plan_create(ctypes.byref(h), sa, ns, ia, ni, mode, out_type, p,
                                         _tune(tune), _stream(stream)), "srng_batch_plan_create")
    return h.value


def srng_batch_plan_launch(plan: int, stream=None) -> None:
    _check(load().srng_batch_plan_launch(plan, _stream(stream)), "srng_batch_plan_launch")


def srng_batch_plan_info(plan: int):
    n = _u64()
    k = _u32()
    _check(load().srng_batch_plan_info(plan, ctypes.byref(n), ctypes.byref(k)), "srng_batch_plan_info")
    return n.value, k.value


def srng_batch_plan_destroy(plan: int) -> None:
    _check(load().srng_batch_plan_destroy(plan), "srng_batch_plan_destroy")


def srng_batch_run(sets, inst, mode: int, out_type: int, out_dev, stream=None) -> None:
    sa, ns = _sets(sets)
    ia, ni = _instances(inst)
    p = _buffer(out_dev, _batch_out_bytes(ia, ni, mode, out_type), "srng_batch_run", "cuda")
    _check(load().srng_batch_run(sa, ns, ia, ni, mode, out_type, p, _stream(stream)), "srng_batch_run")


def srng_batch_run_static(sets, inst, mode: int, out_type: int, out_dev, stream=None) -> None:
    """srng_batch_run without any allocation (fixed scratch inside the library;
    at most 4096 instances and 8 sets; calls that overlap on the GPU race)."""
    sa, ns = _sets(sets)
    ia, ni = _instances(inst)
    p = _buffer(out_dev, _batch_out_bytes(ia, ni, mode, out_type), "srng_batch_run_static", "cuda")
    _check(load().srng_batch_run_static(sa, ns, ia, ni, mode, out_type, p, _stream(stream)),
           "srng_batch_run_static")


# ---------------------------------------------------------------- serving
def srng_server_create(handle: int, cfg=None) -> int:
    c = None
    if cfg is not None:
        c = ctypes.byref(cfg if isinstance(cfg, ServerConfig) else ServerConfig(**cfg))
    h = _vp()
    _check(load().srng_server_create(ctypes.byref(h), handle, c), "srng_server_create")
    return h.value


def srng_server_submit(srv: int, stream: int, n: int, out_type: int) -> int:
    t = _u64()
    _check(load().srng_server_submit(srv, stream, n, out_type, ctypes.byref(t)), "srng_server_submit")
    return t.value


def srng_server_submit_at(srv: int, stream: int, pos: int, n: int, out_type: int) -> int:
    t = _u64()
    _check(load().srng_server_submit_at(srv, stream, pos, n, out_type, ctypes.byref(t)), "srng_server_submit_at")
    return t.value


def srng_server_poll(srv: int, ticket: int):
    done = _int()
    p = _vp()
    _check(load().srng_server_poll(srv, ticket, ctypes.byref(done), ctypes.byref(p)), "srng_server_poll")
    return bool(done.value), p.value


def srng_server_wait(srv: int, ticket: int, timeout_ms: int = 60000) -> int:
    p = _vp()
    _check(load().srng_server_wait(srv, ticket, timeout_ms, ctypes.byref(p)), "srng_server_wait")
    return p.value


def srng_server_release(srv: int, ticket: int) -> None:
    _check(load().srng_server_release(srv, ticket), "srng_server_release")


def srng_server_read(srv: int, ticket: int, dst, dst_is_host: bool) -> None:
    _check(load().srng_server_read(srv, ticket, _ptr(dst), int(bool(dst_is_host))), "srng_server_read")


def srng_server_get_stats(srv: int) -> ServerStats:
    st = ServerStats()
    _check(load().srng_server_get_stats(srv, ctypes.byref(st)), "srng_server_get_stats")
    return st


def srng_server_reset_stats(srv: int) -> None:
    _check(load().srng_server_reset_stats(srv), "srng_server_reset_stats")


def srng_server_destroy(srv: int) -> None:
    _check(load().srng_server_destroy(srv), "srng_server_destroy")


def srng_server_replay(srv: int, requests, out_type: int, time_scale: float = 1.0, timeout_ms: int = 600000):
    """requests: sequence of (arrival_s, stream, n) or Request; returns ServerStats."""
    arr = (Request * len(requests))()
    for i, r in enumerate(requests):
        arr[i] = r if isinstance(r, Request) else Request(*r)
    st = ServerStats()
    _check(load().srng_server_replay(srv, arr, len(requests), out_type, time_scale, timeout_ms, ctypes.byref(st)),
           "srng_server_replay")
    return st

