"""srng_batch_run_static: the batched launch for callers that cannot allocate.

Some callers must not allocate device memory per call -- their device memory
belongs to another allocator, or their loop cannot afford cudaMalloc /
cudaFree.  srng_batch_run_static serves them from a fixed scratch array
inside the library.  These tests call it through the C ABI and check that two
calls in a row give, bit for bit, what the allocating srng_batch_run gives
(the tolerance of every parity test here is zero: outputs are exact
integers or exactly defined floats).  This file is collected last so that a
run stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng

pytestmark = pytest.mark.gpu


def _instances(n, seed):
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, 30000, n)
    lengths[:4] = [0, 1, 2, 3]
    offsets = rng.integers(0, 9, n)
    gens = np.array([i % 2 for i in range(n)])
    outoff = np.zeros(n, dtype=np.uint64)
    outoff[1:] = np.cumsum(lengths[:-1] + (np.arange(n - 1) % 3))  # ragged, unaligned placement
    inst = [srng.Instance(set_index=int(gens[i]), stream=i, offset=int(offsets[i]), length=int(lengths[i]),
                          out_offset=int(outoff[i])) for i in range(n)]
    return inst, int(outoff[-1] + lengths[-1])


@pytest.fixture
def sets():
    hm = srng.srng_create(srng.SRNG_MRG32K3A, 0x5EED5EED5EED5EED, 1024, srng.SRNG_SPACING_STREAM)
    hp = srng.srng_create(srng.SRNG_PHILOX4X32_10, 0xC0FFEE, 1024)
    yield [hm, hp]
    srng.srng_destroy(hm)
    srng.srng_destroy(hp)


@pytest.mark.parametrize("out_type,dtype", [(srng.SRNG_OUT_U32, torch.int32), (srng.SRNG_OUT_F64, torch.float64)])
def test_static_batch_matches_allocating_batch_twice(sets, out_type, dtype):
    inst, total = _instances(300, 21)
    ref = torch.zeros(total, dtype=dtype, device="cuda")
    srng.srng_batch_run(sets, inst, srng.SRNG_BATCH_WRITE, out_type, ref)
    for call in range(2):
        # a fresh zeroed buffer per call: a call that did nothing would leave zeros
        got = torch.zeros(total, dtype=dtype, device="cuda")
        srng.srng_batch_run_static(sets, inst, srng.SRNG_BATCH_WRITE, out_type, got)
        torch.cuda.synchronize()
        bits = torch.int32 if dtype == torch.int32 else torch.int64
        assert torch.equal(got.view(bits), ref.view(bits)), call


def test_static_fused_pi_matches_allocating_batch_twice(sets):
    inst, _ = _instances(1000, 5)
    ref = torch.empty(len(inst), dtype=torch.int64, device="cuda")
    srng.srng_batch_run(sets, inst, srng.SRNG_BATCH_FUSED_PI, srng.SRNG_OUT_U32, ref)
    for call in range(2):
        got = torch.full((len(inst),), -7, dtype=torch.int64, device="cuda")
        srng.srng_batch_run_static(sets, inst, srng.SRNG_BATCH_FUSED_PI, srng.SRNG_OUT_U32, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), call


def test_static_batch_rejects_sizes_beyond_its_maximum(sets):
    inst = [srng.Instance(set_index=0, stream=0, offset=0, length=1, out_offset=i) for i in range(4097)]
    out = torch.empty(4097, dtype=torch.int32, device="cuda")
    with pytest.raises(srng.SrngError) as e:
        srng.srng_batch_run_static(sets, inst, srng.SRNG_BATCH_WRITE, srng.SRNG_OUT_U32, out)
    assert e.value.name == "SRNG_ERR_ARG" and "4096" in str(e.value)
