"""Independent third-party implementations the oracle is pinned against, run
as libraries (nothing of theirs is copied here):

- SplitMix64's output mixer (Stafford's "variant 13" finalizer) from the
  pybind11 headers installed with the Python package ``pybind11``
  (``pybind11::detail::mix64``), compiled into a two-line shim with g++;
- the MT19937 initialisation multiplier (x -> 1812433253 (x ^ (x >> 30)) + i),
  which TinyMT32's seeding also uses, from numpy's legacy MT19937 seeding:
  word 1 of ``RandomState(x)``'s key is 1812433253 (x ^ (x >> 30)) + 1.

Each helper returns None (the test then skips) where the implementation is
not installed.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import sysconfig
import tempfile

_MIX64 = None


def pybind11_mix64():
    """Callable uint64 -> uint64 evaluating pybind11::detail::mix64, or None."""
    global _MIX64
    if _MIX64 is not None:
        return _MIX64 or None
    _MIX64 = False
    try:
        import pybind11
    except ImportError:
        return None
    inc = pybind11.get_include()
    py_inc = sysconfig.get_paths().get("include", "")
    gxx = shutil.which("g++")
    if not gxx or not os.path.exists(os.path.join(inc, "pybind11", "detail", "internals.h")) or \
            not os.path.exists(os.path.join(py_inc, "Python.h")):
        return None
    d = tempfile.mkdtemp(prefix="pin_mix64_")
    src = os.path.join(d, "mix64.cpp")
    so = os.path.join(d, "mix64.so")
    with open(src, "w") as f:
        f.write("#include <pybind11/detail/internals.h>\n"
                "extern \"C\" unsigned long long pin_mix64(unsigned long long z)"
                " { return pybind11::detail::mix64(z); }\n")
    res = subprocess.run([gxx, "-std=c++17", "-O1", "-w", "-shared", "-fPIC", "-I", inc, "-I", py_inc, src,
                          "-o", so], capture_output=True, text=True)
    if res.returncode != 0:
        return None
    lib = ctypes.CDLL(so)
    lib.pin_mix64.restype = ctypes.c_uint64
    lib.pin_mix64.argtypes = [ctypes.c_uint64]
    _MIX64 = lambda z: int(lib.pin_mix64(z & 0xFFFFFFFFFFFFFFFF))
    return _MIX64


def mt19937_init_mix(x: int) -> int:
    """1812433253 * (x ^ (x >> 30)) mod 2^32, read from numpy's MT19937
    legacy seeding (state word 1 after seeding with x is that value + 1)."""
    import numpy as np
    key = np.random.RandomState(int(x) & 0xFFFFFFFF).get_state()[1]
    return (int(key[1]) - 1) & 0xFFFFFFFF
