"""srng_batch_run_static: the batched launch for callers that cannot allocate.

Some callers must not allocate device memory per call -- their device memory
belongs to another allocator, or their loop cannot afford cudaMalloc /
cudaFree.  srng_batch_run_static serves them from a fixed scratch array
inside the library.  These tests call it through the C ABI and check that two
calls in a row give, bit for bit, what the allocating srng_batch_run gives,
and what the CPU oracle gives for sets of every generator and layout the
batch accepts (the tolerance of every parity test here is zero: outputs are
exact integers or exactly defined floats).  They also check that a second call
takes no device memory, and that calls whose work-item counts would overflow
the kernels' 32-bit counters are refused before anything runs.  This file is
collected last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng
from oracle import oracle as O

pytestmark = pytest.mark.gpu

SEED_M, SEED_P = 0x5EED5EED5EED5EED, 0xC0FFEE
TYPES = [(srng.SRNG_OUT_U32, torch.int32), (srng.SRNG_OUT_F32, torch.float32), (srng.SRNG_OUT_F64, torch.float64)]


def _bits(t):
    return t.view(torch.int64 if t.element_size() == 8 else torch.int32)


def _instances(n, seed, n_streams=1024, max_len=30000):
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, max_len, n)
    lengths[:4] = [0, 1, 2, 3]
    offsets = rng.integers(0, 9, n)
    gens = np.array([i % 2 for i in range(n)])
    outoff = np.zeros(n, dtype=np.uint64)
    outoff[1:] = np.cumsum(lengths[:-1] + (np.arange(n - 1) % 3))  # ragged, unaligned placement
    inst = [srng.Instance(set_index=int(gens[i]), stream=i % n_streams, offset=int(offsets[i]),
                          length=int(lengths[i]), out_offset=int(outoff[i])) for i in range(n)]
    return inst, int(outoff[-1] + lengths[-1])


@pytest.fixture
def sets():
    hm = srng.srng_create(srng.SRNG_MRG32K3A, SEED_M, 1024, srng.SRNG_SPACING_STREAM)
    hp = srng.srng_create(srng.SRNG_PHILOX4X32_10, SEED_P, 1024)
    yield [hm, hp]
    srng.srng_destroy(hm)
    srng.srng_destroy(hp)


@pytest.mark.parametrize("out_type,dtype", TYPES)
def test_static_batch_matches_allocating_batch_twice(sets, out_type, dtype):
    inst, total = _instances(300, 21)
    ref = torch.zeros(total, dtype=dtype, device="cuda")
    srng.srng_batch_run(sets, inst, srng.SRNG_BATCH_WRITE, out_type, ref)
    for call in range(2):
        # a fresh zeroed buffer per call: a call that did nothing would leave zeros
        got = torch.zeros(total, dtype=dtype, device="cuda")
        srng.srng_batch_run_static(sets, inst, srng.SRNG_BATCH_WRITE, out_type, got)
        torch.cuda.synchronize()
        assert torch.equal(_bits(got), _bits(ref)), call


def test_static_fused_pi_matches_allocating_batch_twice(sets):
    inst, _ = _instances(1000, 5)
    ref = torch.empty(len(inst), dtype=torch.int64, device="cuda")
    srng.srng_batch_run(sets, inst, srng.SRNG_BATCH_FUSED_PI, srng.SRNG_OUT_U32, ref)
    for call in range(2):
        got = torch.full((len(inst),), -7, dtype=torch.int64, device="cuda")
        srng.srng_batch_run_static(sets, inst, srng.SRNG_BATCH_FUSED_PI, srng.SRNG_OUT_U32, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), call


@pytest.mark.parametrize("mode", [srng.SRNG_BATCH_WRITE, srng.SRNG_BATCH_FUSED_PI])
def test_static_batch_at_its_instance_limit(sets, mode):
    """Exactly SRNG_BATCH_STATIC_MAX_INSTANCES (4096) instances: the prefix-sum
    kernel's last thread then owns the last instances and writes the total."""
    inst, total = _instances(4096, 77, max_len=4000)
    n = len(inst)
    if mode == srng.SRNG_BATCH_WRITE:
        ref = torch.zeros(total, dtype=torch.int32, device="cuda")
        got = torch.zeros(total, dtype=torch.int32, device="cuda")
    else:
        ref = torch.empty(n, dtype=torch.int64, device="cuda")
        got = torch.full((n,), -7, dtype=torch.int64, device="cuda")
    srng.srng_batch_run(sets, inst, mode, srng.SRNG_OUT_U32, ref)
    srng.srng_batch_run_static(sets, inst, mode, srng.SRNG_OUT_U32, got)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    # the last instances, which the scan's last thread covers, also against the oracle
    y0 = O.seed_expand(SEED_M)
    g = got.cpu().numpy()
    for i in range(n - 6, n):
        x = inst[i]
        if x.set_index == 0:
            st = O.mrg_jump(O.mrg_stream_starts(y0, 127, x.stream, 1)[0], x.offset)
            if mode == srng.SRNG_BATCH_WRITE:
                want = O.mrg_generate(st, x.length)[0]
            else:
                want = O.mrg_pi_count(st, x.length)
        else:
            if mode == srng.SRNG_BATCH_WRITE:
                want = O.philox_generate((SEED_P & 0xFFFFFFFF, SEED_P >> 32), x.stream, x.offset, x.length)
            else:
                want = O.philox_pi_count((SEED_P & 0xFFFFFFFF, SEED_P >> 32), x.stream, x.offset, x.length)
        if mode == srng.SRNG_BATCH_WRITE:
            assert np.array_equal(g[x.out_offset:x.out_offset + x.length].view(np.uint32), want), i
        else:
            assert g[i] == want, i


# Eight sets, one of each kind the batch accepts: MRG32k3a streams, substreams
# and a range of streams far from 0; Philox counter split, key per stream and a
# range; Threefry4x32-20 and Threefry4x64-20.
EIGHT = [("mrg_stream", srng.SRNG_MRG32K3A, srng.SRNG_SPACING_STREAM, None),
         ("mrg_substream", srng.SRNG_MRG32K3A, srng.SRNG_SPACING_SUBSTREAM, None),
         ("mrg_range", srng.SRNG_MRG32K3A, srng.SRNG_SPACING_STREAM, 1000),
         ("philox", srng.SRNG_PHILOX4X32_10, srng.SRNG_SPACING_STREAM, None),
         ("philox_keyed", srng.SRNG_PHILOX4X32_10_KEYED, srng.SRNG_SPACING_STREAM, None),
         ("philox_range", srng.SRNG_PHILOX4X32_10, srng.SRNG_SPACING_STREAM, 1 << 40),
         ("threefry", srng.SRNG_THREEFRY4X32_20, srng.SRNG_SPACING_STREAM, None),
         ("threefry64", srng.SRNG_THREEFRY4X64_20, srng.SRNG_SPACING_STREAM, None)]


@pytest.fixture
def eight_sets():
    hs = []
    try:
        for _, gen, spacing, base in EIGHT:
            seed = SEED_M if gen == srng.SRNG_MRG32K3A else SEED_P
            if base is None:
                hs.append(srng.srng_create(gen, seed, 16, spacing))
            else:
                hs.append(srng.srng_create_range(gen, seed, base, 16, spacing))
        yield hs
    finally:
        for h in hs:
            srng.srng_destroy(h)


def _oracle_instance(kind, stream, offset, length, out_type, pi):
    """The oracle's values (or quarter-disc count) for one instance of a set of
    the given kind, from the seed alone."""
    key = (SEED_P & 0xFFFFFFFF, SEED_P >> 32)
    if kind.startswith("mrg"):
        e = 76 if kind == "mrg_substream" else 127
        s = stream + (1000 if kind == "mrg_range" else 0)
        st = O.mrg_stream_starts(O.seed_expand(SEED_M), e, s, 1)[0]
        st = O.mrg_jump(st, offset) if offset else st
        return O.mrg_pi_count(st, length) if pi else O.mrg_generate(st, length, out_type)[0]
    if kind in ("philox", "philox_range"):
        s = stream + ((1 << 40) if kind == "philox_range" else 0)
        return O.philox_pi_count(key, s, offset, length) if pi else O.philox_generate(key, s, offset, length, out_type)
    if kind == "philox_keyed":
        if not pi:
            return O.philox_keyed_generate(SEED_P, stream, offset, length, out_type)
        w = O.philox_keyed_generate(SEED_P, stream, offset, length, O.OUT_U32)
        return sum(O.pi_hit_philox(int(w[2 * k]), int(w[2 * k + 1])) for k in range(length // 2))
    if kind == "threefry":
        return O.threefry_pi_count(SEED_P, stream, offset, length) if pi else \
            O.threefry_generate(SEED_P, stream, offset, length, out_type)
    return O.threefry64_pi_count(SEED_P, stream, offset, length) if pi else \
        O.threefry64_generate(SEED_P, stream, offset, length, out_type)


def _eight_instances():
    rng = np.random.default_rng(1412)
    inst, meta = [], []
    off = 0
    for si, (kind, _, _, _) in enumerate(EIGHT):
        lengths = [0, 1, 7, 4097] + rng.integers(100, 20000, 3).tolist()
        for j, L in enumerate(lengths):
            o = int(rng.integers(0, 9))
            inst.append(srng.Instance(set_index=si, stream=j, offset=o, length=int(L), out_offset=off))
            meta.append((kind, j, o, int(L)))
            off += int(L) + j % 3
    return inst, meta, off


@pytest.mark.parametrize("out_type,dtype", TYPES)
def test_static_batch_of_every_set_kind_equals_oracle(eight_sets, out_type, dtype):
    inst, meta, total = _eight_instances()
    for call in range(2):
        got = torch.zeros(total, dtype=dtype, device="cuda")
        srng.srng_batch_run_static(eight_sets, inst, srng.SRNG_BATCH_WRITE, out_type, got)
        torch.cuda.synchronize()
        g = got.cpu().numpy()
        for x, (kind, s, o, L) in zip(inst, meta):
            want = np.asarray(_oracle_instance(kind, s, o, L, out_type, False))
            have = g[x.out_offset:x.out_offset + L]
            assert np.array_equal(have.view(np.uint64 if dtype == torch.float64 else np.uint32),
                                  want.view(np.uint64 if dtype == torch.float64 else np.uint32)), (call, kind, s, L)


def test_static_fused_pi_of_every_set_kind_equals_oracle(eight_sets):
    inst, meta, _ = _eight_instances()
    for call in range(2):
        got = torch.full((len(inst),), -7, dtype=torch.int64, device="cuda")
        srng.srng_batch_run_static(eight_sets, inst, srng.SRNG_BATCH_FUSED_PI, srng.SRNG_OUT_U32, got)
        torch.cuda.synchronize()
        g = got.cpu().numpy()
        for i, (kind, s, o, L) in enumerate(meta):
            assert g[i] == _oracle_instance(kind, s, o, L, 0, True), (call, kind, s, L)


def test_static_batch_takes_no_device_memory_after_its_first_call(sets):
    """The first call on a device looks up the scratch array; later calls
    allocate nothing: the device's free memory is the same before and after."""
    inst, total = _instances(500, 3)
    out = torch.zeros(total, dtype=torch.int32, device="cuda")
    srng.srng_batch_run_static(sets, inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    srng.srng_batch_run_static(sets, inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_batch_rejects_sizes_beyond_its_maximum(sets):
    inst = [srng.Instance(set_index=0, stream=0, offset=0, length=1, out_offset=i) for i in range(4097)]
    out = torch.empty(4097, dtype=torch.int32, device="cuda")
    with pytest.raises(srng.SrngError) as e:
        srng.srng_batch_run_static(sets, inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, out)
    assert e.value.name == "SRNG_ERR_ARG" and "4096" in str(e.value)


@pytest.mark.parametrize("case", ["mrg_2^42", "mrg_sum", "philox_2^48"])
def test_static_batch_refuses_work_item_overflow_before_launching(sets, case):
    """Work-item counts are 32-bit on the device: an MRG32k3a instance of 2^42
    draws (2^33 chunks), 4096 instances of 2^41 draws (2^39 items) or one
    Philox instance of 2^48 draws (2^35 items) is refused with SRNG_ERR_ARG,
    and the counts buffer is left as it was (nothing was launched)."""
    if case == "mrg_2^42":
        inst = [srng.Instance(set_index=0, stream=0, offset=0, length=1 << 42, out_offset=0)]
    elif case == "mrg_sum":
        inst = [srng.Instance(set_index=0, stream=i % 1024, offset=0, length=1 << 41, out_offset=0)
                for i in range(4096)]
    else:
        inst = [srng.Instance(set_index=1, stream=0, offset=0, length=1 << 48, out_offset=0)]
    counts = torch.full((len(inst),), -7, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(srng.SrngError) as e:
        srng.srng_batch_run_static(sets, inst, srng.SRNG_BATCH_FUSED_PI, srng.SRNG_OUT_U32, counts)
    assert e.value.name == "SRNG_ERR_ARG"
    torch.cuda.synchronize()
    assert bool((counts == -7).all())
