"""The C ABI library loads, exports every declared entry point, and its host
logic (seed expansion, jump matrices, argument validation) agrees with the
oracle -- no GPU needed: none of these calls reach the device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1412_8266_gb300 as srng
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1412_8266_gb300 import _build
    _build.build()
    return srng.load()


def _declared_functions():
    names = set()
    for h in ("srng.h",):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(srng_[a-z_0-9]+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 25, names
    out = subprocess.run(["nm", "-D", "--defined-only", srng.lib_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_python_binding_covers_every_entry_point(lib):
    for n in _declared_functions():
        assert hasattr(srng, n), n


def test_version_and_status_strings(lib):
    assert srng.srng_abi_version() == srng.SRNG_ABI_VERSION == 3
    assert srng.srng_status_string(0) == "SRNG_OK"
    assert srng.srng_status_string(3) == "SRNG_ERR_STATE"


@pytest.mark.parametrize("seed", [0, 1, 0xC0FFEE, 0x5EED5EED5EED5EED, 2**64 - 1])
def test_seed_expansion_matches_oracle(lib, seed):
    assert srng.srng_seed_expand(seed) == [int(x) for x in O.seed_expand(seed)]


@pytest.mark.parametrize("unit,shift", [(srng.SRNG_JUMP_DRAWS, 0), (srng.SRNG_JUMP_SUBSTREAMS, 76),
                                        (srng.SRNG_JUMP_STREAMS, 127)])
def test_jump_matrices_match_oracle(lib, unit, shift):
    rng = np.random.default_rng(1)
    for n in [0, 1, 2, 3, 7, 4096, 2**40 + 17, int(rng.integers(0, 2**63)) * 3 + 1]:
        a1, a2 = srng.srng_jump_matrix(unit, n)
        d = n << shift
        assert a1 == O.mrg_matpow(0, d % (O.M1**3 - 1) if d >= 2**128 else d).tolist()
        assert a2 == O.mrg_matpow(1, d % (O.M2**3 - 1) if d >= 2**128 else d).tolist()


def test_argument_errors_need_no_gpu(lib):
    with pytest.raises(srng.SrngError) as e:
        srng.srng_create(srng.SRNG_MRG32K3A, 1, 0)
    assert e.value.name == "SRNG_ERR_ARG"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_create(7, 1, 10)
    assert e.value.name == "SRNG_ERR_ARG"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_create_from_state([0, 0, 0, 1, 2, 3], 4)
    assert e.value.name == "SRNG_ERR_STATE"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_create_from_state([O.M1, 1, 1, 1, 1, 1], 4)
    assert e.value.name == "SRNG_ERR_STATE"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_generate(0, 0, 1, 1, srng.SRNG_OUT_U32, 0)
    assert e.value.name == "SRNG_ERR_ARG"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_set_tune(srng.SRNG_PHILOX4X32_10, srng.SRNG_OUT_U32, {"unroll": 3})
    assert e.value.name == "SRNG_ERR_ARG"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_set_tune(srng.SRNG_MRG32K3A, srng.SRNG_OUT_U32, {"chunk": 100})
    assert e.value.name == "SRNG_ERR_ARG"
    assert "multiple of 32" in srng.srng_last_error()
    for dist, n, ptr, why in ((5, 4, 64, "distribution"), (srng.SRNG_DIST_NORMAL, 3, 64, "pairs"),
                              (srng.SRNG_DIST_NORMAL, 4, 68, "misaligned"), (srng.SRNG_DIST_EXPONENTIAL, 4, 0, "NULL")):
        with pytest.raises(srng.SrngError) as e:
            srng.srng_transform(dist, ptr, n, ptr)
        assert e.value.name == "SRNG_ERR_ARG" and why in srng.srng_last_error()
    srng.srng_transform(srng.SRNG_DIST_NORMAL, 0, 0, 0)   # empty: nothing to do, no device needed


def test_tune_table_roundtrip(lib):
    srng.srng_set_tune(srng.SRNG_PHILOX4X32_10, srng.SRNG_OUT_F32, {"unroll": 4, "block_threads": 128})
    t = srng.srng_get_tune(srng.SRNG_PHILOX4X32_10, srng.SRNG_OUT_F32)
    assert t.unroll == 4 and t.block_threads == 128
    srng.srng_set_tune(srng.SRNG_PHILOX4X32_10, srng.SRNG_OUT_F32, None)
    t = srng.srng_get_tune(srng.SRNG_PHILOX4X32_10, srng.SRNG_OUT_F32)
    assert t.unroll == 4 and t.block_threads == 256


def test_destroy_null_is_ok(lib):
    srng.srng_destroy(0)


def test_library_has_no_oracle_dependency(lib):
    """The CUDA library must not link or name the oracle."""
    out = subprocess.run(["nm", "-D", srng.lib_path()], capture_output=True, text=True, check=True).stdout
    assert "oracle" not in out
    ldd = subprocess.run(["ldd", srng.lib_path()], capture_output=True, text=True).stdout
    assert "liboracle" not in ldd


def test_range_set_argument_errors(lib):
    with pytest.raises(srng.SrngError) as e:
        srng.srng_create_range(srng.SRNG_MRG32K3A, 1, 2**64 - 3, 5)
    assert e.value.name == "SRNG_ERR_RANGE"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_create_range(srng.SRNG_PHILOX4X32_10, 1, 0, 5, state=[1, 2, 3, 4, 5, 6])
    assert e.value.name == "SRNG_ERR_ARG"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_create_range(srng.SRNG_MRG32K3A, 1, 0, 5, state=[0, 0, 0, 4, 5, 6])
    assert e.value.name == "SRNG_ERR_STATE"


def test_tinymt_parameter_search_matches_oracle(lib):
    """The library's host parameter search (its own Berlekamp-Massey and GF(2)
    arithmetic, threaded) finds the same sets, in the same order, as the
    oracle's plain search."""
    for seed in (0, 0x5EED, 2**64 - 1):
        got = srng.srng_tinymt_find_params(seed, 5)
        assert np.array_equal(got, O.tinymt32_find_params(seed, 5)), seed
    assert srng.srng_tinymt_check_params(0x8F7011EE, 0xFC78FF1F)
    assert not srng.srng_tinymt_check_params(0x8F7011EE, 0xFC78FF1E) or O.tinymt32_max_period(0x8F7011EE, 0xFC78FF1E)
    rng = np.random.default_rng(9)
    for mat1, mat2 in rng.integers(0, 2**32, (64, 2), dtype=np.uint64):
        assert srng.srng_tinymt_check_params(int(mat1), int(mat2)) == O.tinymt32_max_period(int(mat1), int(mat2))


def test_tinymt_arguments_need_no_gpu(lib):
    with pytest.raises(srng.SrngError) as e:
        srng.srng_create_tinymt(np.zeros((0, 3), dtype=np.uint32), 4, 1)
    assert e.value.name == "SRNG_ERR_ARG"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_create_tinymt([[1, 2, 3]], 0, 1)
    assert e.value.name == "SRNG_ERR_ARG"


def test_binding_checks_buffers_before_the_call():
    """The binding refuses a buffer it can see is wrong (too small, strided, on
    the wrong side) before any library call; raw addresses pass through."""
    import torch
    from paper_1412_8266_gb300 import _buffer
    a = np.zeros(10, dtype=np.uint32)
    assert _buffer(a, 40, "f", "host") == a.ctypes.data
    with pytest.raises(ValueError, match="needs 44"):
        _buffer(a, 44, "f", "host")
    with pytest.raises(ValueError, match="contiguous"):
        _buffer(np.zeros((4, 4), dtype=np.uint32)[:, 1], 4, "f", "host")
    with pytest.raises(ValueError, match="CUDA buffer"):
        _buffer(a, 4, "f", "cuda")
    t = torch.zeros(8, dtype=torch.float64)
    assert _buffer(t, 64, "f", "host") == t.data_ptr()
    with pytest.raises(ValueError, match="needs 72"):
        _buffer(t, 72, "f", "any")
    with pytest.raises(ValueError, match="CUDA buffer"):
        _buffer(t, 8, "f", "cuda")
    with pytest.raises(ValueError, match="contiguous"):
        _buffer(torch.zeros(4, 4)[:, 0], 4, "f", "host")
    assert _buffer(12345, 1 << 40, "f", "cuda") == 12345
    assert _buffer(None, 0, "f", "cuda") == 0
