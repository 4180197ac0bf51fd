"""MRG32k3a on the GPU vs the CPU oracle (bit-exact): stream placement (K1),
jumps, bulk generation (K2) and the integer -> uniform conversions (A4)."""
import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng
from oracle import oracle as O
from tests.gpu_util import assert_bitexact, empty, to_np

pytestmark = pytest.mark.gpu
TYPES = [srng.SRNG_OUT_U32, srng.SRNG_OUT_F32, srng.SRNG_OUT_F64]
M1 = O.M1


def get_states(h, begin, count):
    st = np.zeros((count, 6), dtype=np.uint32)
    srng.srng_get_state(h, begin, count, st)
    return st


@pytest.fixture
def sets():
    made = []

    def track(h):
        made.append(h)
        return h

    yield track
    for h in made:
        srng.srng_destroy(h)


@pytest.mark.parametrize("spacing,e", [(srng.SRNG_SPACING_STREAM, 127), (srng.SRNG_SPACING_SUBSTREAM, 76)])
def test_placement_from_state(sets, spacing, e):
    h = sets(srng.srng_create_from_state([12345] * 6, 1000, spacing))
    ref = O.mrg_stream_starts([12345] * 6, e, 0, 1000)
    assert np.array_equal(get_states(h, 0, 1000), ref)


def test_placement_from_seed_large_indices(sets):
    seed = 0x5EED5EED5EED5EED
    n = (1 << 18) + 5
    h = sets(srng.srng_create(srng.SRNG_MRG32K3A, seed, n, srng.SRNG_SPACING_STREAM))
    y0 = O.seed_expand(seed)
    for first in (0, 777, (1 << 17) + 3, n - 40):
        ref = O.mrg_stream_starts(y0, 127, first, 40)
        assert np.array_equal(get_states(h, first, 40), ref), first
    d = srng.srng_describe(h)
    assert list(d.seed_state) == [int(x) for x in y0] and d.n_streams == n


@pytest.mark.parametrize("unit,shift", [(srng.SRNG_JUMP_DRAWS, 0), (srng.SRNG_JUMP_SUBSTREAMS, 76),
                                        (srng.SRNG_JUMP_STREAMS, 127)])
def test_jump_vs_oracle(sets, unit, shift):
    h = sets(srng.srng_create(srng.SRNG_MRG32K3A, 7, 50, srng.SRNG_SPACING_SUBSTREAM))
    before = get_states(h, 0, 50)
    rng = np.random.default_rng(3)
    for n in [1, 2, 3, 1000, int(rng.integers(1, 2**62))]:
        srng.srng_jump(h, 10, 20, unit, n)
        after = get_states(h, 0, 50)
        d = n << shift
        for i in range(50):
            if 10 <= i < 30:
                # each component has period m^3 - 1 (pinned in the oracle tests)
                a = O.mrg_jump(before[i], d % (O.M1**3 - 1))[:3]
                b = O.mrg_jump(before[i], d % (O.M2**3 - 1))[3:]
                want = [int(x) for x in a] + [int(x) for x in b]
            else:
                want = [int(x) for x in before[i]]
            assert [int(x) for x in after[i]] == want, (n, i)
        before = after


@pytest.mark.parametrize("out_type", TYPES)
@pytest.mark.parametrize("S,n", [(1, 1), (1, 3), (5, 31), (5, 32), (7, 33), (2, 4095), (3, 4097), (33, 1000), (1, 200_001)])
def test_small_ragged_vs_oracle(sets, out_type, S, n):
    seed = 12
    h = sets(srng.srng_create(srng.SRNG_MRG32K3A, seed, S + 3, srng.SRNG_SPACING_STREAM))
    starts = get_states(h, 0, S + 3)
    _, out = empty(S * n, out_type)
    srng.srng_generate(h, 3, S, n, out_type, out)
    torch.cuda.synchronize()
    ref, final = O.mrg_bulk(starts[3:], n, out_type)
    assert_bitexact(to_np(out, out_type).reshape(S, n), ref, out_type)
    after = get_states(h, 0, S + 3)
    assert np.array_equal(after[3:], final)
    assert np.array_equal(after[:3], starts[:3])


@pytest.mark.parametrize("out_type", TYPES)
@pytest.mark.parametrize("pad", [1, 2, 3])
@pytest.mark.parametrize("chunk", [32, 96, 256])
def test_chunked_and_unaligned_vs_oracle(sets, out_type, pad, chunk):
    """Streams split into chunks reached by jump-ahead, unaligned outputs."""
    S, n = 6, 3001
    h = sets(srng.srng_create_from_state([1, 2, 3, 4, 5, 6], S, srng.SRNG_SPACING_SUBSTREAM))
    starts = get_states(h, 0, S)
    _, out = empty(S * n, out_type, pad=pad)
    srng.srng_generate_tuned(h, 0, S, n, out_type, out, dict(chunk=chunk))
    torch.cuda.synchronize()
    ref, final = O.mrg_bulk(starts, n, out_type)
    assert_bitexact(to_np(out, out_type).reshape(S, n), ref, out_type)
    assert np.array_equal(get_states(h, 0, S), final)


@pytest.mark.parametrize("n", [4096, 5000])
@pytest.mark.parametrize("tune", [dict(chunk=32), dict(chunk=4096), dict(block_threads=128),
                                  dict(vector_store=2), dict(blocks_per_sm=1, chunk=512),
                                  dict(vector_store=3, chunk=512), dict(vector_store=3, chunk=4096),
                                  dict(vector_store=3, chunk=32, block_threads=128),
                                  dict(vector_store=4, chunk=512), dict(vector_store=4, chunk=4096),
                                  dict(vector_store=4, chunk=32, block_threads=128),
                                  dict(vector_store=4, resident=3), dict(vector_store=1, resident=3),
                                  dict(vector_store=3, resident=32)])
def test_tuning_never_changes_output(sets, tune, n):
    S = 300
    outs = []
    for t in (None, tune):
        h = sets(srng.srng_create(srng.SRNG_MRG32K3A, 77, S))
        o = torch.empty(S * n, dtype=torch.float64, device="cuda")
        srng.srng_generate_tuned(h, 0, S, n, srng.SRNG_OUT_F64, o, t)
        outs.append(o)
    torch.cuda.synchronize()
    assert torch.equal(outs[0].view(torch.int64), outs[1].view(torch.int64))


@pytest.mark.parametrize("out_type,vs", [(srng.SRNG_OUT_U32, 3), (srng.SRNG_OUT_F32, 3), (srng.SRNG_OUT_F64, 3),
                                         (srng.SRNG_OUT_F64, 4)])
@pytest.mark.parametrize("S,n,chunk,extra", [
    (3, 1024, 32, {}),                          # 32 chunks per stream: lane products only
    (5, 6144, 64, dict(block_threads=128)),     # 96 chunks: warp digits 0-2, 4-warp blocks
    (7, 131072, 128, {}),                       # 1024 chunks: warp digits up to 31
    (2, 65536, 32, {}),                         # 2048 chunks: bit 10 of the chunk index
    (1, 131072, 32, {}),                        # 4096 chunks: bits 10 and 11
    (64, 65536, 64, dict(blocks_per_sm=1)),     # more items than threads: grid-stride passes
    (9, 8192, 128, dict(resident=3)),           # shared memory reserved beside the lane table
    (5000, 2048, 64, {}),                       # 160,000 items: many grid-stride passes
])
def test_radix_chunk_starts_vs_oracle(sets, out_type, vs, S, n, chunk, extra):
    """Direct rows with radix-32 chunk starts (chunk count a multiple of 32),
    from the third stream of the set on, against the oracle in full."""
    h = sets(srng.srng_create(srng.SRNG_MRG32K3A, 0xABCDEF, S + 2, srng.SRNG_SPACING_STREAM))
    starts = get_states(h, 0, S + 2)
    _, out = empty(S * n, out_type)
    srng.srng_generate_tuned(h, 2, S, n, out_type, out, dict(chunk=chunk, vector_store=vs, **extra))
    torch.cuda.synchronize()
    ref, final = O.mrg_bulk(starts[2:], n, out_type)
    assert_bitexact(to_np(out, out_type).reshape(S, n), ref, out_type)
    after = get_states(h, 0, S + 2)
    assert np.array_equal(after[2:], final)
    assert np.array_equal(after[:2], starts[:2])


@pytest.mark.parametrize("out_type,tune", [(srng.SRNG_OUT_F64, dict(chunk=64)),   # radix-32 chunk starts
                                           (srng.SRNG_OUT_U32, dict(chunk=64)),
                                           (srng.SRNG_OUT_F64, dict(chunk=4096))])  # one item per stream
def test_graph_replay_of_generate_calls(sets, out_type, tune):
    """Three generation calls captured in one CUDA graph (each a generation
    kernel and its dependent state advance), replayed twice: the buffers hold
    the second replay's draws and the states moved by six calls, as the oracle
    says."""
    S, n, K = 8, 4096, 3
    h = sets(srng.srng_create(srng.SRNG_MRG32K3A, 99, S, srng.SRNG_SPACING_STREAM))
    starts = get_states(h, 0, S)
    bufs = [empty(S * n, out_type)[1] for _ in range(K)]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        srng.srng_generate_tuned(h, 0, S, n, out_type, bufs[0], tune, side)  # warm-up outside the capture
        srng.srng_reset(h, side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        for k in range(K):
            srng.srng_generate_tuned(h, 0, S, n, out_type, bufs[k], tune, side)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    ref, final = O.mrg_bulk(starts, 2 * K * n, out_type)
    for k in range(K):
        want = ref[:, (K + k) * n:(K + k + 1) * n]
        assert_bitexact(to_np(bufs[k], out_type).reshape(S, n), want, out_type)
    assert np.array_equal(get_states(h, 0, S), final)


def test_state_save_restore_resumes(sets):
    """Checkpoint mid-stream, continue, restore, continue again: same draws."""
    h = sets(srng.srng_create(srng.SRNG_MRG32K3A, 5, 10))
    a = torch.empty(10 * 100, dtype=torch.int32, device="cuda")
    srng.srng_generate(h, 0, 10, 100, srng.SRNG_OUT_U32, a)
    saved = get_states(h, 0, 10)
    b1 = torch.empty(10 * 77, dtype=torch.int32, device="cuda")
    srng.srng_generate(h, 0, 10, 77, srng.SRNG_OUT_U32, b1)
    srng.srng_set_state(h, 0, 10, saved)
    b2 = torch.empty(10 * 77, dtype=torch.int32, device="cuda")
    srng.srng_generate(h, 0, 10, 77, srng.SRNG_OUT_U32, b2)
    torch.cuda.synchronize()
    assert torch.equal(b1, b2)
    bad = saved.copy()
    bad[3, 0] = M1
    with pytest.raises(srng.SrngError) as e:
        srng.srng_set_state(h, 0, 10, bad)
    assert e.value.name == "SRNG_ERR_STATE"


def test_full_size_mrg_plain_f64():
    """Whole workload: all-12345 seed state, 64 streams 2^127 apart, 2^16 FP64
    draws each (4M values), compared in full."""
    S, n = 64, 1 << 16
    h = srng.srng_create_from_state([12345] * 6, S, srng.SRNG_SPACING_STREAM)
    try:
        out = torch.empty(S * n, dtype=torch.float64, device="cuda")
        srng.srng_generate(h, 0, S, n, srng.SRNG_OUT_F64, out)
        torch.cuda.synchronize()
        ref, _ = O.mrg_bulk(O.mrg_stream_starts([12345] * 6, 127, 0, S), n, O.OUT_F64)
        assert_bitexact(to_np(out, 2).reshape(S, n), ref, 2)
        v = out.cpu().numpy()
        assert v.min() > 0.0 and v.max() < 1.0
    finally:
        srng.srng_destroy(h)


@pytest.mark.parametrize("tune_u, tune_f", [
    (None, None),  # the built-in shapes
    # the shapes the benchmark's tuner picks at this size (uint32: staged rows,
    # one item per stream; FP64: per-lane rows in items of 2048 draws)
    (dict(block_threads=256, blocks_per_sm=8, chunk=4096, vector_store=1),
     dict(block_threads=256, blocks_per_sm=8, chunk=2048, vector_store=3)),
    (dict(block_threads=128, blocks_per_sm=16, chunk=1024, vector_store=3),
     dict(block_threads=128, blocks_per_sm=16, chunk=4096, vector_store=1)),
    (dict(block_threads=256, blocks_per_sm=8, chunk=4096, vector_store=1),
     dict(block_threads=256, blocks_per_sm=8, chunk=2048, vector_store=4)),
    (dict(block_threads=256, blocks_per_sm=8, chunk=2048, vector_store=3, resident=6),
     dict(block_threads=256, blocks_per_sm=8, chunk=2048, vector_store=4, resident=6)),
    (dict(block_threads=256, blocks_per_sm=32, chunk=1024, vector_store=3, resident=6),
     dict(block_threads=256, blocks_per_sm=16, chunk=1024, vector_store=4, resident=6)),
])
def test_full_size_mrg_bulk_sampled(tune_u, tune_f):
    """Whole workload in the benchmark's launch configurations: seed
    0x5EED5EED5EED5EED, 2^18 streams x 4096 draws, u32 then f64 after a reset.
    1024 sampled streams are compared in full with the oracle; every f64 value
    equals the conversion of the u32 value at the same place; all u32 values
    lie in [1, m1]."""
    seed, S, n = 0x5EED5EED5EED5EED, 1 << 18, 4096
    h = srng.srng_create(srng.SRNG_MRG32K3A, seed, S, srng.SRNG_SPACING_STREAM)
    try:
        starts = get_states(h, 0, S)
        u = torch.empty(S * n, dtype=torch.int32, device="cuda")
        f = torch.empty(S * n, dtype=torch.float64, device="cuda")
        srng.srng_generate_tuned(h, 0, S, n, srng.SRNG_OUT_U32, u, tune_u)
        srng.srng_reset(h)
        srng.srng_generate_tuned(h, 0, S, n, srng.SRNG_OUT_F64, f, tune_f)
        torch.cuda.synchronize()
        rng = np.random.default_rng(11)
        pick = np.unique(np.concatenate([[0, 1, S - 1], rng.integers(0, S, 1021)]))
        ref, _ = O.mrg_bulk(starts[pick], n, O.OUT_U32)
        got = u.view(S, n)[torch.from_numpy(pick).cuda()].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref)
        conv = torch.empty_like(f)
        srng.srng_convert(srng.SRNG_MRG32K3A, srng.SRNG_OUT_F64, u, S * n, conv)
        torch.cuda.synchronize()
        assert torch.equal(conv.view(torch.int64), f.view(torch.int64))
        uu = u.to(torch.int64) & 0xFFFFFFFF
        assert int(uu.min()) >= 1 and int(uu.max()) <= M1
        # states moved by exactly n draws
        after = get_states(h, 0, 64)
        _, final = O.mrg_bulk(starts[:64], n, O.OUT_U32)
        assert np.array_equal(after, final)
    finally:
        srng.srng_destroy(h)


# ------------------------------------------------------------- conversions (A4)
def test_mrg_f64_conversion_exhaustive():
    """The integer-built double equals the IEEE round-to-nearest-even product
    z * norm for every z in [1, m1] (GPU FP64 multiply as the reference), and
    the oracle's multiply on a sample that includes the edges."""
    norm = 1.0 / 4294967088.0
    chunk = 1 << 28
    z0 = 1
    while z0 <= M1:
        cnt = min(chunk, M1 - z0 + 1)
        z = torch.arange(z0, z0 + cnt, dtype=torch.int64, device="cuda")
        zi32 = torch.where(z >= 2**31, z - 2**32, z).to(torch.int32)
        out = torch.empty(cnt, dtype=torch.float64, device="cuda")
        srng.srng_convert(srng.SRNG_MRG32K3A, srng.SRNG_OUT_F64, zi32, cnt, out)
        ref = z.to(torch.float64) * norm
        assert torch.equal(out.view(torch.int64), ref.view(torch.int64)), z0
        z0 += cnt
    rng = np.random.default_rng(2)
    zs = np.concatenate([[1, 2, 3, M1 - 1, M1, (1 << 25) - 1, 1 << 25, (1 << 31) + 7],
                         rng.integers(1, M1 + 1, 1 << 16)]).astype(np.uint32)
    zd = torch.from_numpy(zs.view(np.int32)).cuda()
    out = torch.empty(zs.size, dtype=torch.float64, device="cuda")
    srng.srng_convert(srng.SRNG_MRG32K3A, srng.SRNG_OUT_F64, zd, zs.size, out)
    ref = O.convert(zs, 0, O.OUT_F64)
    assert_bitexact(out.cpu().numpy(), ref, 2)


@pytest.mark.parametrize("gen", [srng.SRNG_MRG32K3A, srng.SRNG_PHILOX4X32_10])
def test_f32_and_philox_f64_conversions_exhaustive(gen):
    """f32 = (v >> 8) 2^-24 and Philox f64 = (w + 1/2) 2^-32 for all 2^32 words."""
    chunk = 1 << 28
    for w0 in range(0, 1 << 32, chunk):
        w = torch.arange(w0, w0 + chunk, dtype=torch.int64, device="cuda")
        w32 = torch.where(w >= 2**31, w - 2**32, w).to(torch.int32)
        f = torch.empty(chunk, dtype=torch.float32, device="cuda")
        srng.srng_convert(gen, srng.SRNG_OUT_F32, w32, chunk, f)
        assert torch.equal(f, (w >> 8).to(torch.float32) * (2.0 ** -24)), w0
        if gen == srng.SRNG_PHILOX4X32_10:
            d = torch.empty(chunk, dtype=torch.float64, device="cuda")
            srng.srng_convert(gen, srng.SRNG_OUT_F64, w32, chunk, d)
            assert torch.equal(d.view(torch.int64), ((w.to(torch.float64) + 0.5) * 2.0 ** -32).view(torch.int64))
    sample = np.array([0, 1, 255, 256, 2**24, 2**31, 2**32 - 1], dtype=np.uint32)
    d = torch.empty(sample.size, dtype=torch.float32, device="cuda")
    srng.srng_convert(gen, srng.SRNG_OUT_F32, torch.from_numpy(sample.view(np.int32)).cuda(), sample.size, d)
    assert_bitexact(d.cpu().numpy(), O.convert(sample, gen, O.OUT_F32), 1)


def test_device_view_exposes_states(sets):
    h = sets(srng.srng_create(srng.SRNG_MRG32K3A, 3, 8))
    v = srng.srng_get_device_view(h)
    assert v.gen == 0 and v.n_streams == 8 and v.mrg_state
    h2 = sets(srng.srng_create(srng.SRNG_PHILOX4X32_10, (5 << 32) | 9, 8))
    v2 = srng.srng_get_device_view(h2)
    assert v2.gen == 1 and v2.key0 == 9 and v2.key1 == 5 and v2.philox_pos


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("gen", [srng.SRNG_MRG32K3A, srng.SRNG_PHILOX4X32_10])
def test_generate_into_host_memory(gen, pinned):
    """srng_generate_host (pinned: direct kernel stores over the host link;
    pageable: staged pieces and copies) equals srng_generate on the device,
    also when one stream is longer than a staging piece."""
    S, n = 3, (70 << 20) // 3 + 5  # 3 streams x ~23M f64 > one 256 MiB piece per stream
    ha = srng.srng_create(gen, 31, S)
    hb = srng.srng_create(gen, 31, S)
    try:
        dev = torch.empty(S * n, dtype=torch.float64, device="cuda")
        srng.srng_generate(ha, 0, S, n, srng.SRNG_OUT_F64, dev)
        if pinned:
            host = torch.empty(S * n, dtype=torch.float64, pin_memory=True)
        else:
            host = np.empty(S * n, dtype=np.float64)
        srng.srng_generate_host(hb, 0, S, n, srng.SRNG_OUT_F64, host)
        got = host.numpy() if pinned else host
        assert np.array_equal(got.view(np.uint64), dev.cpu().numpy().view(np.uint64))
        # both sets moved by n draws
        if gen == srng.SRNG_MRG32K3A:
            assert np.array_equal(get_states(ha, 0, S), get_states(hb, 0, S))
    finally:
        srng.srng_destroy(ha)
        srng.srng_destroy(hb)


# ------------------------------------------------------------- stream ranges
@pytest.mark.parametrize("base,spacing,e", [(1 << 40, srng.SRNG_SPACING_STREAM, 127),
                                            (2**64 - 8, srng.SRNG_SPACING_STREAM, 127),
                                            (123456789, srng.SRNG_SPACING_SUBSTREAM, 76)])
def test_range_set_places_far_streams(base, spacing, e):
    """A set holding streams [base, base + 8): far stream numbers (up to the
    paper's 2^64 - 1) without the streams below them."""
    seed = 0x5EED5EED5EED5EED
    h = srng.srng_create_range(srng.SRNG_MRG32K3A, seed, base, 8, spacing)
    try:
        st = get_states(h, 0, 8)
        ref = O.mrg_stream_starts(O.seed_expand(seed), e, base, 8)
        assert np.array_equal(st, ref)
        assert srng.srng_describe(h).stream_base == base
        out = torch.empty(8 * 1000, dtype=torch.int32, device="cuda")
        srng.srng_generate(h, 0, 8, 1000, srng.SRNG_OUT_U32, out)
        torch.cuda.synchronize()
        want, _ = O.mrg_bulk(ref, 1000, O.OUT_U32)
        assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(8, 1000), want)
    finally:
        srng.srng_destroy(h)


def test_range_set_equals_slice_of_full_set():
    full = srng.srng_create_from_state([12345] * 6, 100, srng.SRNG_SPACING_STREAM)
    part = srng.srng_create_range(srng.SRNG_MRG32K3A, 0, 60, 40, srng.SRNG_SPACING_STREAM, state=[12345] * 6)
    try:
        assert np.array_equal(get_states(full, 60, 40), get_states(part, 0, 40))
    finally:
        srng.srng_destroy(full)
        srng.srng_destroy(part)


@pytest.mark.parametrize("gen", [srng.SRNG_PHILOX4X32_10, srng.SRNG_PHILOX4X32_10_KEYED])
def test_philox_range_set_top_stream_numbers(gen):
    seed, base, n = 0x0123456789ABCDEF, 2**64 - 5, 777
    h = srng.srng_create_range(gen, seed, base, 5, srng.SRNG_SPACING_STREAM)
    try:
        out = torch.empty(5 * n, dtype=torch.int32, device="cuda")
        srng.srng_generate(h, 0, 5, n, srng.SRNG_OUT_U32, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32).reshape(5, n)
        for i in range(5):
            if gen == srng.SRNG_PHILOX4X32_10:
                ref = O.philox_generate((seed & 0xFFFFFFFF, seed >> 32), base + i, 0, n)
            else:
                ref = O.philox_keyed_generate(seed, base + i, 0, n)
            assert np.array_equal(got[i], ref), i
        # batch and server on the range set use the same stream numbers
        inst = [srng.Instance(set_index=0, stream=i, offset=3, length=100, out_offset=100 * i) for i in range(5)]
        b = torch.zeros(500, dtype=torch.int32, device="cuda")
        srng.srng_batch_run([h], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, b)
        bb = b.cpu().numpy().view(np.uint32).reshape(5, 100)
        for i in range(5):
            if gen == srng.SRNG_PHILOX4X32_10:
                ref = O.philox_generate((seed & 0xFFFFFFFF, seed >> 32), base + i, n + 3, 100)
            else:
                ref = O.philox_keyed_generate(seed, base + i, n + 3, 100)
            assert np.array_equal(bb[i], ref), i
    finally:
        srng.srng_destroy(h)
