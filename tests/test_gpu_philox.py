"""Philox4x32-10 bulk generation on the GPU vs the CPU oracle (bit-exact)."""
import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng
from oracle import oracle as O
from tests.gpu_util import assert_bitexact, empty, key_of, to_np

pytestmark = pytest.mark.gpu
TYPES = [srng.SRNG_OUT_U32, srng.SRNG_OUT_F32, srng.SRNG_OUT_F64]


@pytest.fixture
def philox_set():
    made = []

    def make(seed, n_streams):
        h = srng.srng_create(srng.SRNG_PHILOX4X32_10, seed, n_streams)
        made.append(h)
        return h

    yield make
    for h in made:
        srng.srng_destroy(h)


@pytest.mark.parametrize("out_type", TYPES)
@pytest.mark.parametrize("n_streams,n", [(1, 1), (1, 3), (3, 4), (7, 5), (2, 4095), (3, 4097), (5, 1000), (1, 70001)])
def test_small_ragged_vs_oracle(philox_set, out_type, n_streams, n):
    seed = 0x0123456789ABCDEF
    h = philox_set(seed, n_streams + 2)
    _, out = empty(n_streams * n, out_type)
    srng.srng_generate(h, 2, n_streams, n, out_type, out)
    torch.cuda.synchronize()
    ref, pos = O.philox_bulk(key_of(seed), 2, [0] * n_streams, n, out_type)
    assert_bitexact(to_np(out, out_type).reshape(n_streams, n), ref, out_type)
    got_pos = np.zeros(n_streams + 2, dtype=np.uint64)
    srng.srng_get_state(h, 0, n_streams + 2, got_pos)
    assert list(got_pos) == [0, 0] + [n] * n_streams


@pytest.mark.parametrize("out_type", TYPES)
@pytest.mark.parametrize("start", [1, 2, 3, 5, 6])
@pytest.mark.parametrize("pad", [0, 1, 3])
def test_unaligned_positions_and_outputs(philox_set, out_type, start, pad):
    """Start positions not on a Philox block, output pointers not 16-byte aligned."""
    seed = 0xC0FFEE
    S, n = 4, 1027
    h = philox_set(seed, S)
    srng.srng_jump(h, 0, S, srng.SRNG_JUMP_DRAWS, start)
    srng.srng_jump(h, 1, 1, srng.SRNG_JUMP_DRAWS, 2)  # streams at different alignments
    _, out = empty(S * n, out_type, pad=pad)
    srng.srng_generate(h, 0, S, n, out_type, out)
    torch.cuda.synchronize()
    pos = [start, start + 2, start, start]
    ref, _ = O.philox_bulk(key_of(seed), 0, pos, n, out_type)
    assert_bitexact(to_np(out, out_type).reshape(S, n), ref, out_type)


def test_successive_calls_continue_the_stream(philox_set):
    seed = 99
    h = philox_set(seed, 3)
    a = torch.empty(3 * 333, dtype=torch.int32, device="cuda")
    b = torch.empty(3 * 334, dtype=torch.int32, device="cuda")
    srng.srng_generate(h, 0, 3, 333, srng.SRNG_OUT_U32, a)
    srng.srng_generate(h, 0, 3, 334, srng.SRNG_OUT_U32, b)
    torch.cuda.synchronize()
    got = np.concatenate([to_np(a, 0).reshape(3, 333), to_np(b, 0).reshape(3, 334)], axis=1)
    ref, _ = O.philox_bulk(key_of(seed), 0, [0, 0, 0], 667, O.OUT_U32)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("tune", [dict(unroll=1), dict(unroll=4), dict(block_threads=128, unroll=2),
                                  dict(vector_store=2), dict(blocks_per_sm=1), dict(block_threads=64, unroll=4)])
def test_tuning_never_changes_output(philox_set, tune):
    seed = 0xC0FFEE
    S, n = 3, 100_003
    outs = []
    for t in (None, tune):
        h = philox_set(seed, S)
        o = torch.empty(S * n, dtype=torch.float32, device="cuda")
        srng.srng_generate_tuned(h, 0, S, n, srng.SRNG_OUT_F32, o, t)
        outs.append(o)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])


def test_full_size_philox_bulk_sampled():
    """Full workload: key 0xC0FFEE, counters 0..2^28-1 (2^30 words), u32 and
    f32, in the launch configuration the benchmark uses.  Sampled positions
    and both ends are checked against the oracle word by word; f32 is checked
    against the u32 run at every position."""
    seed, n = 0xC0FFEE, 1 << 30
    h = srng.srng_create(srng.SRNG_PHILOX4X32_10, seed, 1)
    try:
        u = torch.empty(n, dtype=torch.int32, device="cuda")
        f = torch.empty(n, dtype=torch.float32, device="cuda")
        srng.srng_generate(h, 0, 1, n, srng.SRNG_OUT_U32, u)
        srng.srng_reset(h)
        srng.srng_generate(h, 0, 1, n, srng.SRNG_OUT_F32, f)
        torch.cuda.synchronize()
        key = key_of(seed)
        rng = np.random.default_rng(5)
        idx = np.concatenate([np.arange(4096), np.arange(n - 4096, n), rng.integers(0, n, 4096)])
        got = u[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint32)
        ref = np.array([O.philox_word(key, 0, int(i)) for i in idx], dtype=np.uint32)
        assert np.array_equal(got, ref)
        # f32 == (u32 >> 8) 2^-24 everywhere, computed in exact integer/float ops on the GPU
        uu = u.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        expect = ((uu >> 8).to(torch.float32)) * (2.0 ** -24)
        assert torch.equal(expect, f)
        pos = np.zeros(1, dtype=np.uint64)
        srng.srng_get_state(h, 0, 1, pos)
        assert int(pos[0]) == n
    finally:
        srng.srng_destroy(h)


@pytest.mark.parametrize("gen", [srng.SRNG_PHILOX4X32_10, srng.SRNG_PHILOX4X32_10_KEYED])
@pytest.mark.parametrize("tune", [None, dict(unroll=2)])
def test_full_size_many_streams_sampled(gen, tune):
    """The many-short-streams workload at full size: 2^18 streams x 4096 words
    (the flat kernel, a run of block pairs per lane), then every stream moved 3
    draws on and 4096 more words from there (unaligned starts).  Sampled
    streams and both ends are compared with the oracle in full; every
    position moved by 4096 + 3 + 4096."""
    seed, S, n = 0xC0FFEE, 1 << 18, 4096
    h = srng.srng_create(gen, seed, S)
    try:
        out = torch.empty(S * n, dtype=torch.int32, device="cuda")
        rng = np.random.default_rng(8)
        pick = np.unique(np.concatenate([[0, 1, S - 1], rng.integers(0, S, 253)]))
        sel = torch.from_numpy(pick).cuda()
        for start in (0, n + 3):
            if start:
                srng.srng_jump(h, 0, S, srng.SRNG_JUMP_DRAWS, 3)
            srng.srng_generate_tuned(h, 0, S, n, srng.SRNG_OUT_U32, out, tune)
            torch.cuda.synchronize()
            got = out.view(S, n)[sel].cpu().numpy().view(np.uint32)
            if gen == srng.SRNG_PHILOX4X32_10:
                ref = np.stack([O.philox_generate(key_of(seed), int(s), start, n) for s in pick])
            else:
                ref = np.stack([O.philox_keyed_generate(seed, int(s), start, n) for s in pick])
            assert np.array_equal(got, ref), start
        pos = np.zeros(S, dtype=np.uint64)
        srng.srng_get_state(h, 0, S, pos)
        assert np.all(pos == 2 * n + 3)
    finally:
        srng.srng_destroy(h)


def test_position_overflow_is_rejected(philox_set):
    h = philox_set(1, 1)
    srng.srng_jump(h, 0, 1, srng.SRNG_JUMP_DRAWS, 2**64 - 10)
    with pytest.raises(srng.SrngError) as e:
        srng.srng_generate(h, 0, 1, 11, srng.SRNG_OUT_U32, torch.empty(11, dtype=torch.int32, device="cuda"))
    assert e.value.name == "SRNG_ERR_RANGE"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_jump(h, 0, 1, srng.SRNG_JUMP_SUBSTREAMS, 1)
    assert e.value.name == "SRNG_ERR_UNSUPPORTED"


def test_empty_and_range_edges(philox_set):
    h = philox_set(1, 4)
    srng.srng_generate(h, 0, 0, 10, srng.SRNG_OUT_U32, 0)
    srng.srng_generate(h, 4, 0, 10, srng.SRNG_OUT_U32, 0)
    srng.srng_generate(h, 0, 4, 0, srng.SRNG_OUT_U32, 0)
    with pytest.raises(srng.SrngError) as e:
        srng.srng_generate(h, 3, 2, 10, srng.SRNG_OUT_U32, torch.empty(20, dtype=torch.int32, device="cuda"))
    assert e.value.name == "SRNG_ERR_RANGE"


# ------------------------------------------------------------- keyed layout
@pytest.mark.parametrize("out_type", TYPES)
@pytest.mark.parametrize("n_streams,n,start", [(1, 5, 0), (7, 4097, 0), (33, 1000, 3), (5, 70001, 6)])
def test_keyed_layout_vs_oracle(philox_set, out_type, n_streams, n, start):
    """Key per stream (Sec. 4.3): key = stream index, counter words 2-3 = seed."""
    seed = 0x0123456789ABCDEF
    h = srng.srng_create(srng.SRNG_PHILOX4X32_10_KEYED, seed, n_streams + 2)
    try:
        assert srng.srng_describe(h).gen == srng.SRNG_PHILOX4X32_10_KEYED
        v = srng.srng_get_device_view(h)
        assert v.flags & 1
        if start:
            srng.srng_jump(h, 0, n_streams + 2, srng.SRNG_JUMP_DRAWS, start)
        _, out = empty(n_streams * n, out_type, pad=1 if start else 0)
        srng.srng_generate(h, 2, n_streams, n, out_type, out)
        torch.cuda.synchronize()
        ref = np.stack([O.philox_keyed_generate(seed, 2 + i, start, n, out_type) for i in range(n_streams)])
        assert_bitexact(to_np(out, out_type).reshape(n_streams, n), ref, out_type)
    finally:
        srng.srng_destroy(h)


def test_keyed_layout_differs_from_counter_split():
    a = srng.srng_create(srng.SRNG_PHILOX4X32_10, 7, 4)
    b = srng.srng_create(srng.SRNG_PHILOX4X32_10_KEYED, 7, 4)
    try:
        x = torch.empty(4 * 64, dtype=torch.int32, device="cuda")
        y = torch.empty(4 * 64, dtype=torch.int32, device="cuda")
        srng.srng_generate(a, 0, 4, 64, srng.SRNG_OUT_U32, x)
        srng.srng_generate(b, 0, 4, 64, srng.SRNG_OUT_U32, y)
        torch.cuda.synchronize()
        assert not torch.equal(x, y)
    finally:
        srng.srng_destroy(a)
        srng.srng_destroy(b)


def test_keyed_layout_in_batch_and_server():
    seed = 0xC0FFEE
    h = srng.srng_create(srng.SRNG_PHILOX4X32_10_KEYED, seed, 50)
    try:
        lengths = [0, 1, 5, 1000, 40001, 7]
        offs = [0, 3, 1, 0, 2, 5]
        outoff = np.concatenate([[0], np.cumsum(lengths[:-1])]).astype(int)
        inst = [srng.Instance(set_index=0, stream=10 + i, offset=offs[i], length=lengths[i],
                              out_offset=int(outoff[i])) for i in range(len(lengths))]
        out = torch.zeros(sum(lengths), dtype=torch.int32, device="cuda")
        srng.srng_batch_run([h], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, out)
        got = out.cpu().numpy().view(np.uint32)
        for i, L in enumerate(lengths):
            ref = O.philox_keyed_generate(seed, 10 + i, offs[i], L)
            assert np.array_equal(got[outoff[i]:outoff[i] + L], ref), i
        static = torch.zeros(sum(lengths), dtype=torch.int32, device="cuda")
        srng.srng_batch_run_static([h], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, static)
        torch.cuda.synchronize()
        assert torch.equal(static, out)
        srv = srng.srng_server_create(h, dict(budget_bytes=16 << 20))
        try:
            t1 = srng.srng_server_submit(srv, 3, 12345, srng.SRNG_OUT_U32)
            t2 = srng.srng_server_submit(srv, 3, 999, srng.SRNG_OUT_U32)
            for t, pos, n in ((t1, 0, 12345), (t2, 12345, 999)):
                srng.srng_server_wait(srv, t, 60000)
                host = np.empty(n, dtype=np.uint32)
                srng.srng_server_read(srv, t, host, True)
                assert np.array_equal(host, O.philox_keyed_generate(seed, 3, pos, n))
                srng.srng_server_release(srv, t)
        finally:
            srng.srng_server_destroy(srv)
    finally:
        srng.srng_destroy(h)
