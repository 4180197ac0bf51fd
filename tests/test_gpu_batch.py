"""Batched instances (persistent graph-captured launch) and the fused Monte
Carlo consumer vs the CPU oracle and vs per-instance plain launches."""
import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng
from oracle import oracle as O
from paper_1412_8266_gb300 import workload as W
from tests.gpu_util import assert_bitexact, empty, key_of, to_np

pytestmark = pytest.mark.gpu
TYPES = [srng.SRNG_OUT_U32, srng.SRNG_OUT_F32, srng.SRNG_OUT_F64]
MRG_SEED, PHX_SEED = 0x5EED5EED5EED5EED, 0xC0FFEE


def _states(h, n):
    st = np.zeros((n, 6), dtype=np.uint32)
    srng.srng_get_state(h, 0, n, st)
    return st


def _make(n_inst, lengths, offsets=None, pad_out=0, gens=None):
    gens = np.array([i % 2 for i in range(n_inst)]) if gens is None else np.asarray(gens)
    lengths = np.asarray(lengths, dtype=np.uint64)
    offsets = np.zeros(n_inst, dtype=np.uint64) if offsets is None else np.asarray(offsets, dtype=np.uint64)
    outoff = np.zeros(n_inst, dtype=np.uint64)
    outoff[1:] = np.cumsum(lengths[:-1] + pad_out)
    inst = [srng.Instance(set_index=int(g), stream=i, offset=int(offsets[i]), length=int(lengths[i]),
                          out_offset=int(outoff[i])) for i, g in enumerate(gens)]
    return gens, lengths, offsets, outoff, inst


def _oracle(gens, lengths, offsets, outoff, mrg_states, mode, out_type, total=None):
    n = len(gens)
    mst = np.zeros((n, 6), dtype=np.uint32)
    for i in range(n):
        if gens[i] == 0:
            mst[i] = O.mrg_jump(mrg_states[i], int(offsets[i])) if offsets[i] else mrg_states[i]
    return O.batch(gens, mst, key_of(PHX_SEED), list(range(n)), offsets, lengths, outoff, mode, out_type,
                   total=total)


@pytest.fixture
def two_sets():
    n = 64
    hm = srng.srng_create(srng.SRNG_MRG32K3A, MRG_SEED, n, srng.SRNG_SPACING_STREAM)
    hp = srng.srng_create(srng.SRNG_PHILOX4X32_10, PHX_SEED, n)
    yield hm, hp, _states(hm, n)
    srng.srng_destroy(hm)
    srng.srng_destroy(hp)


@pytest.mark.parametrize("out_type", TYPES)
@pytest.mark.parametrize("pad_out", [0, 1])
def test_small_mixed_batch_write(two_sets, out_type, pad_out):
    hm, hp, mst = two_sets
    rng = np.random.default_rng(4)
    n = 41
    lengths = rng.integers(0, 9000, n)
    lengths[:6] = [0, 1, 2, 3, 4, 5]
    offsets = rng.integers(0, 7, n)
    gens, lengths, offsets, outoff, inst = _make(n, lengths, offsets, pad_out)
    total = int(outoff[-1] + lengths[-1])
    _, out = empty(total, out_type)
    out.zero_()
    srng.srng_batch_run([hm, hp], inst, srng.SRNG_BATCH_WRITE, out_type, out)
    ref = _oracle(gens, lengths, offsets, outoff, mst, 0, out_type, total=total)
    assert_bitexact(to_np(out, out_type), ref, out_type)


def test_small_mixed_batch_fused_pi(two_sets):
    hm, hp, mst = two_sets
    rng = np.random.default_rng(8)
    n = 50
    lengths = rng.integers(0, 20000, n)
    lengths[:5] = [0, 1, 2, 3, 7]
    offsets = rng.integers(0, 9, n)  # odd offsets exercise unaligned Philox pairs
    gens, lengths, offsets, outoff, inst = _make(n, lengths, offsets)
    counts = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    srng.srng_batch_run([hm, hp], inst, srng.SRNG_BATCH_FUSED_PI, srng.SRNG_OUT_U32, counts)
    ref = _oracle(gens, lengths, offsets, outoff, mst, 1, 0)
    assert np.array_equal(counts.cpu().numpy(), ref)


@pytest.mark.parametrize("tune", [dict(chunk=32, lane_blocks=1), dict(chunk=2048, lane_blocks=512),
                                  dict(blocks_per_sm=1)])
def test_plan_is_graph_replayable_and_tuning_invariant(two_sets, tune):
    hm, hp, mst = two_sets
    lengths = np.arange(1, 61) * 997
    gens, lengths, offsets, outoff, inst = _make(60, lengths)
    total = int(outoff[-1] + lengths[-1])
    a = torch.zeros(total, dtype=torch.int32, device="cuda")
    b = torch.zeros(total, dtype=torch.int32, device="cuda")
    plan = srng.srng_batch_plan_create([hm, hp], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, a)
    plan2 = srng.srng_batch_plan_create([hm, hp], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, b, tune)
    try:
        for _ in range(3):
            srng.srng_batch_plan_launch(plan)
            srng.srng_batch_plan_launch(plan2)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        items, kernels = srng.srng_batch_plan_info(plan)
        assert items > 0 and kernels == 2   # one persistent kernel per generator family present
    finally:
        srng.srng_batch_plan_destroy(plan)
        srng.srng_batch_plan_destroy(plan2)
    ref = _oracle(gens, lengths, offsets, outoff, mst, 0, 0, total=total)
    assert np.array_equal(to_np(a, 0), ref)


def test_full_size_batched_vs_plain_and_oracle():
    """The batched workload at full size (10^4 instances, lengths log-uniform
    in [1e2, 1e7], even = MRG32k3a, odd = Philox), u32 WRITE mode in one
    persistent graph launch: equal to one plain srng_generate per instance on
    fresh sets (whole output compared on the GPU), 24 sampled instances equal
    to the oracle, and the fused counts equal the oracle on the sampled
    instances and estimate pi."""
    gens, lengths, outoff = W.batched_instances()
    n = len(gens)
    total = int(outoff[-1] + lengths[-1])
    hm = srng.srng_create(srng.SRNG_MRG32K3A, MRG_SEED, n, srng.SRNG_SPACING_STREAM)
    hp = srng.srng_create(srng.SRNG_PHILOX4X32_10, PHX_SEED, n)
    try:
        mst = _states(hm, n)
        inst = [srng.Instance(set_index=int(gens[i]), stream=i, offset=0, length=int(lengths[i]),
                              out_offset=int(outoff[i])) for i in range(n)]
        out = torch.zeros(total, dtype=torch.int32, device="cuda")  # padding between slots stays 0
        plan = srng.srng_batch_plan_create([hm, hp], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, out)
        srng.srng_batch_plan_launch(plan)
        torch.cuda.synchronize()
        srng.srng_batch_plan_destroy(plan)
        # plain per-instance launches
        plain = torch.zeros(total, dtype=torch.int32, device="cuda")
        for i in range(n):
            h = hm if gens[i] == 0 else hp
            o = int(outoff[i])
            srng.srng_generate(h, i, 1, int(lengths[i]), srng.SRNG_OUT_U32, plain[o:o + int(lengths[i])])
        torch.cuda.synchronize()
        assert torch.equal(out, plain)
        del plain
        rng = np.random.default_rng(9)
        small = [i for i in range(n) if lengths[i] < 300_000]
        pick = sorted(set(rng.choice(small, 20, replace=False).tolist() + [int(np.argmax(lengths)), 0, 1, n - 1]))
        for i in pick:
            L, o = int(lengths[i]), int(outoff[i])
            got = out[o:o + L].cpu().numpy().view(np.uint32)
            if gens[i] == 0:
                ref, _ = O.mrg_generate(mst[i], L)
            else:
                ref = O.philox_generate(key_of(PHX_SEED), i, 0, L)
            assert np.array_equal(got, ref), i
        del out
        # fused consumer
        srng.srng_reset(hm)
        srng.srng_reset(hp)
        counts = torch.empty(n, dtype=torch.int64, device="cuda")
        plan = srng.srng_batch_plan_create([hm, hp], inst, srng.SRNG_BATCH_FUSED_PI, srng.SRNG_OUT_U32, counts)
        srng.srng_batch_plan_launch(plan)
        torch.cuda.synchronize()
        srng.srng_batch_plan_destroy(plan)
        c = counts.cpu().numpy()
        for i in pick[:12]:
            want = O.mrg_pi_count(mst[i], int(lengths[i])) if gens[i] == 0 else \
                O.philox_pi_count(key_of(PHX_SEED), i, 0, int(lengths[i]))
            assert c[i] == want, i
        pairs = int(np.sum(lengths // 2))
        est = 4.0 * c.sum() / pairs
        assert abs(est - np.pi) < 5 * 4 * np.sqrt(np.pi / 4 * (1 - np.pi / 4) / pairs)
    finally:
        srng.srng_destroy(hm)
        srng.srng_destroy(hp)


@pytest.mark.parametrize("gen", [srng.SRNG_MRG32K3A, srng.SRNG_PHILOX4X32_10])
def test_single_family_plan_has_one_kernel(gen):
    """A batch of one generator family captures one persistent kernel; its
    output equals the oracle's."""
    seed = MRG_SEED if gen == srng.SRNG_MRG32K3A else PHX_SEED
    h = srng.srng_create(gen, seed, 16)
    try:
        lengths = [5, 0, 4097, 70001, 33]
        outoff = np.concatenate([[0], np.cumsum(lengths[:-1])]).astype(int)
        inst = [srng.Instance(set_index=0, stream=i, offset=0, length=L, out_offset=int(outoff[i]))
                for i, L in enumerate(lengths)]
        out = torch.zeros(sum(lengths), dtype=torch.int32, device="cuda")
        plan = srng.srng_batch_plan_create([h], inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, out)
        try:
            srng.srng_batch_plan_launch(plan)
            torch.cuda.synchronize()
            items, kernels = srng.srng_batch_plan_info(plan)
            assert items > 0 and kernels == 1
        finally:
            srng.srng_batch_plan_destroy(plan)
        got = out.cpu().numpy().view(np.uint32)
        if gen == srng.SRNG_MRG32K3A:
            st = _states(h, 16)
            for i, L in enumerate(lengths):
                ref, _ = O.mrg_generate(st[i], L)
                assert np.array_equal(got[outoff[i]:outoff[i] + L], ref), i
        else:
            for i, L in enumerate(lengths):
                assert np.array_equal(got[outoff[i]:outoff[i] + L], O.philox_generate(key_of(PHX_SEED), i, 0, L)), i
    finally:
        srng.srng_destroy(h)
