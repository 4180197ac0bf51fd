"""TinyMT32 (Sec. 4.2: one parameter set per group of streams, 2^64-spaced
substreams within a group) on the GPU vs the CPU oracle, bit for bit:
placement, generation (one item per stream, and chunked streams reached by
Horner jumps), state advance, jumps, state I/O, explicit parameter sets,
and the rejections of the batch and server paths."""
import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng
from oracle import oracle as O
from tests.gpu_util import assert_bitexact, empty, to_np

pytestmark = pytest.mark.gpu
TYPES = [srng.SRNG_OUT_U32, srng.SRNG_OUT_F32, srng.SRNG_OUT_F64]
TMT = srng.SRNG_TINYMT32
SEED = 0x0123456789ABCDEF


def _starts(seed, n_streams, group_size=256):
    ng = (n_streams + group_size - 1) // group_size
    prm = O.tinymt32_find_params(seed, ng)
    return prm, O.tinymt32_stream_starts(seed & 0xFFFFFFFF, prm, group_size, n_streams)


def _states(h, n):
    st = np.zeros((n, 4), dtype=np.uint32)
    srng.srng_get_state(h, 0, n, st)
    return st


@pytest.fixture
def tmt_set():
    made = []

    def make(seed, n_streams):
        h = srng.srng_create(TMT, seed, n_streams)
        made.append(h)
        return h

    yield make
    for h in made:
        srng.srng_destroy(h)


def test_placement_matches_oracle(tmt_set):
    n = 1000   # four groups of 256, the last partial
    h = tmt_set(SEED, n)
    prm, st = _starts(SEED, n)
    assert np.array_equal(_states(h, n), st)
    v = srng.srng_get_device_view(h)
    assert v.gen == TMT and v.tinymt_group_size == 256
    assert srng.srng_describe(h).gen == TMT


@pytest.mark.parametrize("out_type", TYPES)
@pytest.mark.parametrize("n_streams,n", [(1, 1), (3, 5), (300, 4097), (1000, 33), (2, 100001), (5, 70000)])
def test_generate_vs_oracle(tmt_set, out_type, n_streams, n):
    h = tmt_set(SEED, n_streams + 2)
    prm, st = _starts(SEED, n_streams + 2)
    _, out = empty(n_streams * n, out_type)
    srng.srng_generate(h, 1, n_streams, n, out_type, out)
    torch.cuda.synchronize()
    ref, end = O.tinymt32_bulk(st[1:1 + n_streams], prm, 256, n, out_type) if n_streams + 2 <= 256 else \
        _bulk_any_groups(st, prm, 1, n_streams, n, out_type)
    assert_bitexact(to_np(out, out_type).reshape(n_streams, n), ref, out_type)
    got_st = _states(h, n_streams + 2)
    assert np.array_equal(got_st[1:1 + n_streams], end)
    assert np.array_equal(got_st[0], st[0]) and np.array_equal(got_st[-1], st[-1])


def _bulk_any_groups(st, prm, first, count, n, out_type):
    """Oracle bulk output of streams [first, first + count) that span groups."""
    outs, ends = [], []
    for i in range(first, first + count):
        o, e = O.tinymt32_generate(st[i], prm[i // 256], n, out_type)
        outs.append(o)
        ends.append(e)
    return np.stack(outs), np.stack(ends)


@pytest.mark.parametrize("pad", [1, 3])
def test_unaligned_output(tmt_set, pad):
    h = tmt_set(7, 9)
    prm, st = _starts(7, 9)
    _, out = empty(9 * 1001, srng.SRNG_OUT_U32, pad=pad)
    srng.srng_generate(h, 0, 9, 1001, srng.SRNG_OUT_U32, out)
    torch.cuda.synchronize()
    ref, _ = O.tinymt32_bulk(st, prm, 256, 1001)
    assert np.array_equal(to_np(out, 0).reshape(9, 1001), ref)


def test_chunked_equals_one_item_per_stream(tmt_set):
    """A user chunk forces Horner jumps to chunk starts; the output is unchanged."""
    outs = []
    for tune in (None, dict(chunk=4096), dict(chunk=512), dict(chunk=32)):
        h = tmt_set(99, 4)
        o = torch.empty(4 * 20000, dtype=torch.int32, device="cuda")
        srng.srng_generate_tuned(h, 0, 4, 20000, srng.SRNG_OUT_U32, o, tune)
        outs.append((o, _states(h, 4)))
    torch.cuda.synchronize()
    for o, s in outs[1:]:
        assert torch.equal(o, outs[0][0]) and np.array_equal(s, outs[0][1])


def test_successive_calls_and_jump(tmt_set):
    h = tmt_set(5, 3)
    prm, st = _starts(5, 3)
    a = torch.empty(3 * 333, dtype=torch.int32, device="cuda")
    srng.srng_generate(h, 0, 3, 333, srng.SRNG_OUT_U32, a)
    srng.srng_jump(h, 0, 3, srng.SRNG_JUMP_DRAWS, 10**6)
    b = torch.empty(3 * 77, dtype=torch.int32, device="cuda")
    srng.srng_generate(h, 0, 3, 77, srng.SRNG_OUT_U32, b)
    torch.cuda.synchronize()
    for i in range(3):
        p = prm[0]
        first, s1 = O.tinymt32_generate(st[i], p, 333)
        s2 = O.tinymt32_jump(s1, int(p[0]), int(p[1]), 10**6)
        second, _ = O.tinymt32_generate(s2, p, 77)
        assert np.array_equal(to_np(a, 0).reshape(3, 333)[i], first)
        assert np.array_equal(to_np(b, 0).reshape(3, 77)[i], second)
    with pytest.raises(srng.SrngError) as e:
        srng.srng_jump(h, 0, 1, srng.SRNG_JUMP_STREAMS, 1)
    assert e.value.name == "SRNG_ERR_UNSUPPORTED"
    srng.srng_jump(h, 1, 1, srng.SRNG_JUMP_DRAWS, 3 * 2**64 + 5)
    got = _states(h, 3)[1]
    p = prm[0]
    _, s1 = O.tinymt32_generate(st[1], p, 333)
    s1 = O.tinymt32_jump(s1, int(p[0]), int(p[1]), 10**6 + 77)
    assert np.array_equal(got, O.tinymt32_jump(s1, int(p[0]), int(p[1]), 3 * 2**64 + 5))


def test_reset_and_state_io(tmt_set):
    h = tmt_set(11, 40)
    _, st = _starts(11, 40)
    o = torch.empty(40 * 10, dtype=torch.int32, device="cuda")
    srng.srng_generate(h, 0, 40, 10, srng.SRNG_OUT_U32, o)
    srng.srng_reset(h)
    assert np.array_equal(_states(h, 40), st)
    new = st[::-1].copy()
    srng.srng_set_state(h, 0, 40, new)
    assert np.array_equal(_states(h, 40), new)
    with pytest.raises(srng.SrngError) as e:
        srng.srng_set_state(h, 3, 1, np.array([[0x80000000, 0, 0, 0]], dtype=np.uint32))
    assert e.value.name == "SRNG_ERR_STATE"


def test_explicit_parameter_sets():
    prm = O.tinymt32_find_params(0xABC, 3)
    h = srng.srng_create_tinymt(prm, 5, 0xDEADBEEF12345678)
    try:
        st = O.tinymt32_stream_starts(0x12345678, prm, 5, 15)
        assert np.array_equal(_states(h, 15), st)
        o = torch.empty(15 * 1000, dtype=torch.float32, device="cuda")
        srng.srng_generate(h, 0, 15, 1000, srng.SRNG_OUT_F32, o)
        torch.cuda.synchronize()
        ref = np.stack([O.tinymt32_generate(st[i], prm[i // 5], 1000, O.OUT_F32)[0] for i in range(15)])
        assert_bitexact(o.cpu().numpy().reshape(15, 1000), ref, srng.SRNG_OUT_F32)
    finally:
        srng.srng_destroy(h)
    bad = prm.copy()
    bad[1, 1] ^= 1
    if not O.tinymt32_max_period(int(bad[1, 0]), int(bad[1, 1])):
        with pytest.raises(srng.SrngError) as e:
            srng.srng_create_tinymt(bad, 5, 1)
        assert e.value.name == "SRNG_ERR_ARG"


def test_full_size_sampled():
    """2^18 streams x 4096 uint32 (the bulk shape): placement of sampled
    streams and their whole rows against the oracle."""
    S, n = 1 << 18, 4096
    h = srng.srng_create(TMT, SEED, S)
    try:
        out = torch.empty(S * n, dtype=torch.int32, device="cuda")
        srng.srng_generate(h, 0, S, n, srng.SRNG_OUT_U32, out)
        torch.cuda.synchronize()
        rng = np.random.default_rng(3)
        pick = np.unique(np.concatenate([[0, 1, 255, 256, S - 1], rng.integers(0, S, 40)]))
        groups = sorted({int(i) // 256 for i in pick})
        prm_all = srng.srng_tinymt_find_params(SEED, S // 256)
        assert np.array_equal(prm_all[:4], O.tinymt32_find_params(SEED, 4))
        rows = out.view(S, n)[torch.from_numpy(pick).cuda()].cpu().numpy().view(np.uint32)
        for r, i in zip(rows, pick):
            g = int(i) // 256
            p = prm_all[g]
            s0 = O.tinymt32_stream_start(SEED & 0xFFFFFFFF, p, int(i) % 256)
            ref, _ = O.tinymt32_generate(s0, p, n)
            assert np.array_equal(r, ref), (i, g, groups[:3])
    finally:
        srng.srng_destroy(h)


def test_batch_and_server_reject_tinymt(tmt_set):
    h = tmt_set(1, 8)
    inst = [srng.Instance(set_index=0, stream=0, offset=0, length=10, out_offset=0)]
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    for fn in (srng.srng_batch_run, srng.srng_batch_run_static):
        with pytest.raises(srng.SrngError) as e:
            fn([h], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, out)
        assert e.value.name == "SRNG_ERR_UNSUPPORTED"
    with pytest.raises(srng.SrngError) as e:
        srng.srng_server_create(h, dict(budget_bytes=1 << 20))
    assert e.value.name == "SRNG_ERR_UNSUPPORTED"
