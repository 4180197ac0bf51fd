"""Exponential and normal (Box-Muller) variates on the GPU vs the CPU oracle,
bit for bit: exhaustively over all 2^24 FP32 uniforms, from both generators'
FP32 output, in place, on ragged sizes, and through the device header."""
import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng
from oracle import oracle as O
from tests.gpu_util import assert_bitexact, key_of

pytestmark = pytest.mark.gpu
F32 = srng.SRNG_OUT_F32
ALL_U = (np.arange(1 << 24, dtype=np.float64) * 2.0**-24).astype(np.float32)


def _run(dist, u_np, inplace=False, offset=0):
    """offset > 0 places input and output `offset` floats past a 256-byte
    boundary (offset 2: 8-byte aligned, not 16: the scalar kernel)."""
    n = u_np.size
    xb = torch.empty(n + offset, dtype=torch.float32, device="cuda")
    x = xb[offset:]
    x.copy_(torch.from_numpy(np.ascontiguousarray(u_np)))
    y = x if inplace else torch.empty(n + offset, dtype=torch.float32, device="cuda")[offset:]
    srng.srng_transform(dist, x, n, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def test_exponential_every_uniform():
    assert_bitexact(_run(srng.SRNG_DIST_EXPONENTIAL, ALL_U), O.transform(O.DIST_EXPONENTIAL, ALL_U), F32)


def test_normal_every_uniform_in_both_slots():
    """Pairs (u0, u1) = (k, perm(k)) 2^-24: every FP32 uniform appears once as
    the radius input and once as the angle input."""
    perm = np.random.default_rng(3).permutation(1 << 24)
    u = np.empty(2 << 24, dtype=np.float32)
    u[0::2] = ALL_U
    u[1::2] = ALL_U[perm]
    assert_bitexact(_run(srng.SRNG_DIST_NORMAL, u), O.transform(O.DIST_NORMAL, u), F32)


@pytest.mark.parametrize("dist", [srng.SRNG_DIST_EXPONENTIAL, srng.SRNG_DIST_NORMAL])
@pytest.mark.parametrize("n", [2, 4, 6, 1000, 65538, 1000002, 2 * 4 * 152 * 8 * 256 + 6])
@pytest.mark.parametrize("offset", [0, 2])
def test_ragged_sizes_and_in_place(dist, n, offset):
    u = np.random.default_rng(n).integers(0, 1 << 24, n).astype(np.float64) * 2.0**-24
    u = u.astype(np.float32)
    ref = O.transform(dist, u)
    assert_bitexact(_run(dist, u, offset=offset), ref, F32, "out of place")
    assert_bitexact(_run(dist, u, inplace=True, offset=offset), ref, F32, "in place")


def test_exponential_odd_length():
    u = ALL_U[12345:12345 + 1001]
    assert_bitexact(_run(srng.SRNG_DIST_EXPONENTIAL, u), O.transform(O.DIST_EXPONENTIAL, u), F32)


@pytest.mark.parametrize("gen", [srng.SRNG_MRG32K3A, srng.SRNG_PHILOX4X32_10])
def test_from_generated_uniforms(gen):
    """Generator FP32 output -> normals, against the oracle's uniforms -> oracle normals."""
    seed, S, n = 0xC0FFEE, 5, 100_002
    h = srng.srng_create(gen, seed, S)
    try:
        u = torch.empty(S * n, dtype=torch.float32, device="cuda")
        srng.srng_generate(h, 0, S, n, F32, u)
        z = torch.empty_like(u)
        srng.srng_transform(srng.SRNG_DIST_NORMAL, u, u.numel(), z)
        torch.cuda.synchronize()
        if gen == srng.SRNG_MRG32K3A:
            ref_u, _ = O.mrg_bulk(O.mrg_stream_starts(O.seed_expand(seed), 127, 0, S), n, O.OUT_F32)
        else:
            ref_u, _ = O.philox_bulk(key_of(seed), 0, [0] * S, n, O.OUT_F32)
        assert_bitexact(u.cpu().numpy(), ref_u.ravel(), F32, "uniforms")
        assert_bitexact(z.cpu().numpy(), O.transform(O.DIST_NORMAL, ref_u.ravel()), F32, "normals")
    finally:
        srng.srng_destroy(h)


def test_full_size_sampled():
    """2^30 normals from 2^30 Philox uniforms (the bulk workload's size):
    sampled pairs at both ends and at random against the oracle."""
    n = 1 << 30
    h = srng.srng_create(srng.SRNG_PHILOX4X32_10, 0xC0FFEE, 1)
    try:
        u = torch.empty(n, dtype=torch.float32, device="cuda")
        srng.srng_generate(h, 0, 1, n, F32, u)
        srng.srng_transform(srng.SRNG_DIST_NORMAL, u, n, u)   # in place
        torch.cuda.synchronize()
        rng = np.random.default_rng(11)
        pairs = np.concatenate([np.arange(2048), np.arange(n // 2 - 2048, n // 2), rng.integers(0, n // 2, 4096)])
        idx = np.stack([2 * pairs, 2 * pairs + 1], axis=1).ravel()
        got = u[torch.from_numpy(idx).cuda()].cpu().numpy()
        key = key_of(0xC0FFEE)
        words = np.array([O.philox_word(key, 0, int(i)) for i in idx], dtype=np.uint32)
        uni = np.array([O.to_f32(int(w)) for w in words], dtype=np.float32)
        assert_bitexact(got, O.transform(O.DIST_NORMAL, uni), F32)
    finally:
        srng.srng_destroy(h)


def test_odd_normal_length_and_misalignment_rejected():
    x = torch.zeros(9, dtype=torch.float32, device="cuda")
    with pytest.raises(srng.SrngError) as e:
        srng.srng_transform(srng.SRNG_DIST_NORMAL, x, 3, x)
    assert e.value.name == "SRNG_ERR_ARG"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_transform(srng.SRNG_DIST_NORMAL, x[1:], 4, x[1:])
    assert e.value.name == "SRNG_ERR_ARG"
    srng.srng_transform(srng.SRNG_DIST_EXPONENTIAL, x[1:], 7, x[1:])   # 4-byte alignment suffices
