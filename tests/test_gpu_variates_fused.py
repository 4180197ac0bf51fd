"""Fused variate outputs of the bulk generation calls (SRNG_OUT_EXP_F32,
SRNG_OUT_NORMAL_F32) vs the oracle's transforms of the oracle's FP32
uniforms, bit for bit, for every generator and generation kernel."""
import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng
from oracle import oracle as O
from tests.gpu_util import key_of

pytestmark = pytest.mark.gpu
EXP, NORM = srng.SRNG_OUT_EXP_F32, srng.SRNG_OUT_NORMAL_F32
SEED = 0xC0FFEE


def _bits(t):
    return t.detach().cpu().numpy().view(np.uint32)


def _gen(h, b, c, n, out_type, tune=None, pad=0):
    buf = torch.empty(c * n + pad, dtype=torch.float32, device="cuda")
    out = buf[pad:]
    srng.srng_generate_tuned(h, b, c, n, out_type, out, tune)
    torch.cuda.synchronize()
    return _bits(out).reshape(c, n)


def _counter_ref(gen_fn, stream, p, n, out_type):
    """Oracle for the counter-based generators: pairs are absolute positions."""
    p0 = p & ~1
    m = ((p + n + 1) & ~1) - p0
    u = gen_fn(stream, p0, m)
    v = O.transform(O.DIST_NORMAL if out_type == NORM else O.DIST_EXPONENTIAL, u)
    return v[p - p0:p - p0 + n].view(np.uint32)


@pytest.mark.parametrize("gen", [srng.SRNG_PHILOX4X32_10, srng.SRNG_PHILOX4X32_10_KEYED, srng.SRNG_THREEFRY4X32_20,
                                 srng.SRNG_THREEFRY4X64_20])
@pytest.mark.parametrize("out_type", [EXP, NORM])
@pytest.mark.parametrize("S,n,start", [(3, 1000, 0), (4, 1027, 1), (2, 4097, 2), (5, 33, 3), (600, 64, 5),
                                       (1, 70001, 0)])
@pytest.mark.parametrize("tune", [None, dict(unroll=1), dict(vector_store=2)])
def test_counter_based(gen, out_type, S, n, start, tune):
    h = srng.srng_create(gen, SEED, S)
    try:
        if start:
            srng.srng_jump(h, 0, S, srng.SRNG_JUMP_DRAWS, start)
        got = _gen(h, 0, S, n, out_type, tune, pad=1 if start & 1 else 0)
        if gen == srng.SRNG_PHILOX4X32_10:
            fn = lambda s, p, m: O.philox_generate(key_of(SEED), s, p, m, O.OUT_F32)
        elif gen == srng.SRNG_PHILOX4X32_10_KEYED:
            fn = lambda s, p, m: O.philox_keyed_generate(SEED, s, p, m, O.OUT_F32)
        elif gen == srng.SRNG_THREEFRY4X32_20:
            fn = lambda s, p, m: O.threefry_generate(SEED, s, p, m, O.OUT_F32)
        else:
            fn = lambda s, p, m: O.threefry64_generate(SEED, s, p, m, O.OUT_F32)
        for i in range(S):
            assert np.array_equal(got[i], _counter_ref(fn, i, start, n, out_type)), i
    finally:
        srng.srng_destroy(h)


@pytest.mark.parametrize("out_type", [EXP, NORM])
@pytest.mark.parametrize("S,n", [(3, 4096), (7, 1000), (300, 64), (2, 70000)])
@pytest.mark.parametrize("tune", [None, dict(vector_store=1, chunk=512), dict(vector_store=2),
                                  dict(vector_store=3, chunk=1024), dict(chunk=32)])
def test_mrg32k3a(out_type, S, n, tune):
    h = srng.srng_create(srng.SRNG_MRG32K3A, SEED, S)
    try:
        got = _gen(h, 0, S, n, out_type, tune)
        u, _ = O.mrg_bulk(O.mrg_stream_starts(O.seed_expand(SEED), 127, 0, S), n, O.OUT_F32)
        dist = O.DIST_NORMAL if out_type == NORM else O.DIST_EXPONENTIAL
        for i in range(S):
            assert np.array_equal(got[i], O.transform(dist, u[i]).view(np.uint32)), i
    finally:
        srng.srng_destroy(h)


@pytest.mark.parametrize("out_type", [EXP, NORM])
@pytest.mark.parametrize("S,n,tune", [(3, 4096, None), (300, 64, None), (2, 70000, None), (4, 20000, dict(chunk=512)),
                                      (9, 1002, None)])
def test_tinymt32(out_type, S, n, tune):
    h = srng.srng_create(srng.SRNG_TINYMT32, SEED, S)
    try:
        got = _gen(h, 0, S, n, out_type, tune, pad=1)
        prm = O.tinymt32_find_params(SEED, (S + 255) // 256)
        u, _ = O.tinymt32_bulk(O.tinymt32_stream_starts(SEED & 0xFFFFFFFF, prm, 256, S), prm, 256, n, O.OUT_F32)
        dist = O.DIST_NORMAL if out_type == NORM else O.DIST_EXPONENTIAL
        for i in range(S):
            assert np.array_equal(got[i], O.transform(dist, u[i]).view(np.uint32)), i
    finally:
        srng.srng_destroy(h)


def test_state_based_normals_need_even_n_and_streams_continue():
    for gen in (srng.SRNG_MRG32K3A, srng.SRNG_TINYMT32):
        h = srng.srng_create(gen, 1, 2)
        try:
            with pytest.raises(srng.SrngError) as e:
                srng.srng_generate(h, 0, 2, 7, NORM, torch.empty(14, dtype=torch.float32, device="cuda"))
            assert e.value.name == "SRNG_ERR_ARG"
            # normals advance the streams exactly like uniforms
            a = torch.empty(2 * 100, dtype=torch.float32, device="cuda")
            srng.srng_generate(h, 0, 2, 100, NORM, a)
            b = torch.empty(2 * 10, dtype=torch.int32, device="cuda")
            srng.srng_generate(h, 0, 2, 10, srng.SRNG_OUT_U32, b)
            srng.srng_reset(h)
            c = torch.empty(2 * 110, dtype=torch.int32, device="cuda")
            srng.srng_generate(h, 0, 2, 110, srng.SRNG_OUT_U32, c)
            torch.cuda.synchronize()
            assert torch.equal(b.view(2, 10), c.view(2, 110)[:, 100:])
        finally:
            srng.srng_destroy(h)


def test_host_buffer_and_rejections():
    h = srng.srng_create(srng.SRNG_PHILOX4X32_10, SEED, 3)
    try:
        host = np.empty(3 * 5000, dtype=np.float32)
        srng.srng_generate_host(h, 0, 3, 5000, NORM, host)
        for i in range(3):
            ref = _counter_ref(lambda s, p, m: O.philox_generate(key_of(SEED), s, p, m, O.OUT_F32), i, 0, 5000, NORM)
            assert np.array_equal(host.view(np.uint32).reshape(3, 5000)[i], ref)
        inst = [srng.Instance(set_index=0, stream=0, offset=0, length=10, out_offset=0)]
        with pytest.raises(srng.SrngError):
            srng.srng_batch_run([h], inst, srng.SRNG_BATCH_WRITE, NORM, torch.zeros(16, device="cuda"))
    finally:
        srng.srng_destroy(h)
