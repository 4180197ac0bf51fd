"""Threefry4x32-20 and Threefry4x64-20 (Sec. 4.3, key per stream) on the GPU
vs the CPU oracle, bit for bit: bulk generation (both kernels: per-stream
tiles and the flat many-stream kernel), unaligned positions and outputs --
for the 4x64 form, runs that start inside a block of eight words and pairs of
four-word groups that straddle two blocks --, stream ranges, batches (graph
plan, static, fused Monte Carlo) and the server."""
import ctypes
import os

import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng
from oracle import oracle as O
from tests.gpu_util import assert_bitexact, empty, to_np

pytestmark = pytest.mark.gpu
TYPES = [srng.SRNG_OUT_U32, srng.SRNG_OUT_F32, srng.SRNG_OUT_F64]
SEED = 0x0123456789ABCDEF


class _Ref:
    def __init__(self, gen, bulk, generate, word, pi):
        self.gen, self.bulk, self.generate, self.word, self.pi = gen, bulk, generate, word, pi


REFS = {
    "4x32": _Ref(srng.SRNG_THREEFRY4X32_20, O.threefry_bulk, O.threefry_generate, O.threefry_word,
                 O.threefry_pi_count),
    "4x64": _Ref(srng.SRNG_THREEFRY4X64_20, O.threefry64_bulk, O.threefry64_generate, O.threefry64_word,
                 O.threefry64_pi_count),
}


@pytest.fixture(params=sorted(REFS))
def ref(request):
    return REFS[request.param]


@pytest.fixture
def tf_set(ref):
    made = []

    def make(seed, n_streams):
        h = srng.srng_create(ref.gen, seed, n_streams)
        made.append(h)
        return h

    yield make
    for h in made:
        srng.srng_destroy(h)


def test_describe_and_view(tf_set, ref):
    h = tf_set(SEED, 3)
    assert srng.srng_describe(h).gen == ref.gen
    v = srng.srng_get_device_view(h)
    assert v.gen == ref.gen and v.key0 == SEED & 0xFFFFFFFF and v.key1 == SEED >> 32


@pytest.mark.parametrize("out_type", TYPES)
@pytest.mark.parametrize("n_streams,n", [(1, 1), (1, 3), (3, 4), (7, 5), (2, 4095), (3, 4097), (300, 64),
                                         (1000, 33), (1, 70001)])
def test_bulk_vs_oracle(tf_set, ref, out_type, n_streams, n):
    h = tf_set(SEED, n_streams + 2)
    _, out = empty(n_streams * n, out_type)
    srng.srng_generate(h, 2, n_streams, n, out_type, out)
    torch.cuda.synchronize()
    want, _ = ref.bulk(SEED, 2, [0] * n_streams, n, out_type)
    assert_bitexact(to_np(out, out_type).reshape(n_streams, n), want, out_type)
    pos = np.zeros(n_streams + 2, dtype=np.uint64)
    srng.srng_get_state(h, 0, n_streams + 2, pos)
    assert list(pos) == [0, 0] + [n] * n_streams


@pytest.mark.parametrize("out_type", TYPES)
@pytest.mark.parametrize("start,pad", [(1, 0), (2, 1), (3, 3), (6, 0), (4, 0), (9, 2), (12, 1), (15, 0)])
def test_unaligned_positions_and_outputs(tf_set, ref, out_type, start, pad):
    S, n = 4, 1027
    h = tf_set(0xC0FFEE, S)
    srng.srng_jump(h, 0, S, srng.SRNG_JUMP_DRAWS, start)
    srng.srng_jump(h, 1, 1, srng.SRNG_JUMP_DRAWS, 2)
    _, out = empty(S * n, out_type, pad=pad)
    srng.srng_generate(h, 0, S, n, out_type, out)
    torch.cuda.synchronize()
    want, _ = ref.bulk(0xC0FFEE, 0, [start, start + 2, start, start], n, out_type)
    assert_bitexact(to_np(out, out_type).reshape(S, n), want, out_type)


@pytest.mark.parametrize("tune", [dict(unroll=1), dict(unroll=4), dict(vector_store=2), dict(block_threads=64)])
def test_tuning_never_changes_output(tf_set, tune):
    outs = []
    for t in (None, tune):
        h = tf_set(7, 3)
        o = torch.empty(3 * 100_003, dtype=torch.float32, device="cuda")
        srng.srng_generate_tuned(h, 0, 3, 100_003, srng.SRNG_OUT_F32, o, t)
        outs.append(o)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("n_streams,n,start", [(1000, 33, 0), (2000, 16, 5), (513, 100, 4), (4096, 8, 1)])
def test_many_short_streams(tf_set, ref, n_streams, n, start):
    """The flat many-stream kernel, including starts inside a block."""
    h = tf_set(SEED, n_streams)
    srng.srng_jump(h, 0, n_streams, srng.SRNG_JUMP_DRAWS, start)
    out = torch.empty(n_streams * n, dtype=torch.int32, device="cuda")
    srng.srng_generate(h, 0, n_streams, n, srng.SRNG_OUT_U32, out)
    torch.cuda.synchronize()
    want, _ = ref.bulk(SEED, 0, [start] * n_streams, n)
    assert np.array_equal(to_np(out, 0).reshape(n_streams, n), want)


def test_range_set_holds_far_streams(ref):
    base = 2**64 - 10
    h = srng.srng_create_range(ref.gen, SEED, base, 10)
    try:
        out = torch.empty(10 * 9, dtype=torch.int32, device="cuda")
        srng.srng_generate(h, 0, 10, 9, srng.SRNG_OUT_U32, out)
        torch.cuda.synchronize()
        want, _ = ref.bulk(SEED, base, [0] * 10, 9)
        assert np.array_equal(to_np(out, 0).reshape(10, 9), want)
    finally:
        srng.srng_destroy(h)


def test_full_size_sampled(ref):
    """2^30 words of one stream (the bulk size), sampled against the oracle."""
    n = 1 << 30
    h = srng.srng_create(ref.gen, 0xC0FFEE, 1)
    try:
        u = torch.empty(n, dtype=torch.int32, device="cuda")
        srng.srng_generate(h, 0, 1, n, srng.SRNG_OUT_U32, u)
        torch.cuda.synchronize()
        rng = np.random.default_rng(5)
        idx = np.concatenate([np.arange(4096), np.arange(n - 4096, n), rng.integers(0, n, 4096)])
        got = u[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint32)
        want = np.array([ref.word(0xC0FFEE, 0, int(i)) for i in idx], dtype=np.uint32)
        assert np.array_equal(got, want)
    finally:
        srng.srng_destroy(h)


def _instances(lengths, offs, streams, set_index=0):
    outoff = np.concatenate([[0], np.cumsum(lengths[:-1])]).astype(int)
    inst = [srng.Instance(set_index=set_index, stream=int(streams[i]), offset=int(offs[i]), length=int(lengths[i]),
                          out_offset=int(outoff[i])) for i in range(len(lengths))]
    return inst, outoff


def test_batches_and_fused_pi(ref):
    h = srng.srng_create(ref.gen, SEED, 64)
    hm = srng.srng_create(srng.SRNG_MRG32K3A, 1, 64)
    try:
        srng.srng_jump(h, 5, 1, srng.SRNG_JUMP_DRAWS, 3)
        lengths = np.array([0, 1, 5, 1000, 40001, 7, 123457, 2, 3])
        offs = np.array([0, 3, 1, 0, 2, 5, 0, 1, 9])
        streams = np.array([5, 10, 11, 12, 13, 14, 15, 16, 17])
        inst, outoff = _instances(lengths, offs, streams)
        base_pos = {5: 3}
        refs = [ref.generate(SEED, int(streams[i]), base_pos.get(int(streams[i]), 0) + int(offs[i]),
                                    int(lengths[i])) for i in range(len(lengths))]
        out = torch.zeros(int(lengths.sum()), dtype=torch.int32, device="cuda")
        srng.srng_batch_run([h, hm], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, out)
        got = out.cpu().numpy().view(np.uint32)
        for i, L in enumerate(lengths):
            assert np.array_equal(got[outoff[i]:outoff[i] + L], refs[i]), i
        static = torch.zeros_like(out)
        srng.srng_batch_run_static([h, hm], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, static)
        torch.cuda.synchronize()
        assert torch.equal(static, out)
        counts = torch.zeros(len(inst), dtype=torch.int64, device="cuda")
        for t in (None, dict(lane_blocks=3), dict(lane_blocks=128)):
            plan = srng.srng_batch_plan_create([h, hm], inst, srng.SRNG_BATCH_FUSED_PI, srng.SRNG_OUT_U32, counts, t)
            try:
                srng.srng_batch_plan_launch(plan)
                torch.cuda.synchronize()
            finally:
                srng.srng_batch_plan_destroy(plan)
            want = [ref.pi(SEED, int(streams[i]), base_pos.get(int(streams[i]), 0) + int(offs[i]),
                                        int(lengths[i])) for i in range(len(lengths))]
            assert counts.cpu().tolist() == want, t
    finally:
        srng.srng_destroy(h)
        srng.srng_destroy(hm)


def test_server(ref):
    h = srng.srng_create(ref.gen, SEED, 8)
    try:
        srv = srng.srng_server_create(h, dict(budget_bytes=16 << 20))
        try:
            t1 = srng.srng_server_submit(srv, 3, 12345, srng.SRNG_OUT_F64)
            t2 = srng.srng_server_submit(srv, 3, 999, srng.SRNG_OUT_F64)
            for t, pos, n in ((t1, 0, 12345), (t2, 12345, 999)):
                srng.srng_server_wait(srv, t, 60000)
                host = np.empty(n, dtype=np.float64)
                srng.srng_server_read(srv, t, host, True)
                assert np.array_equal(host, ref.generate(SEED, 3, pos, n, O.OUT_F64))
                srng.srng_server_release(srv, t)
        finally:
            srng.srng_server_destroy(srv)
    finally:
        srng.srng_destroy(h)
