"""The library's first draws of every generator against the stored oracle
fixtures (tests/golden/oracle_fixtures.json, written from the oracle alone),
bit for bit."""
import json
import os

import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng
from tests.gpu_util import to_np

pytestmark = pytest.mark.gpu

with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_fixtures.json")) as _f:
    FIX = json.load(_f)
N, S = FIX["draws_per_stream"], FIX["streams"]


def _draw(h, out_type=srng.SRNG_OUT_U32):
    dt = torch.float64 if out_type == srng.SRNG_OUT_F64 else torch.int32
    out = torch.empty(S * N, dtype=dt, device="cuda")
    srng.srng_generate(h, 0, S, N, out_type, out)
    torch.cuda.synchronize()
    return to_np(out, out_type).reshape(S, N)


@pytest.mark.parametrize("name", ["mrg32k3a_12345_streams", "mrg32k3a_12345_substreams", "mrg32k3a_seed_streams"])
def test_mrg32k3a(name):
    c = FIX["cases"][name]
    spacing = srng.SRNG_SPACING_STREAM if c["spacing_log2"] == 127 else srng.SRNG_SPACING_SUBSTREAM
    for out_type, key in ((srng.SRNG_OUT_U32, "u32"), (srng.SRNG_OUT_F64, "f64")):
        if name == "mrg32k3a_seed_streams":
            h = srng.srng_create(srng.SRNG_MRG32K3A, 0x5EED5EED5EED5EED, S, spacing)
        else:
            h = srng.srng_create_from_state(c["seed_state"], S, spacing)
        try:
            got = _draw(h, out_type)
            want = np.array(c[key], dtype=np.uint32 if key == "u32" else np.float64)
            if key == "u32":
                assert np.array_equal(got, want)
            else:
                assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
        finally:
            srng.srng_destroy(h)


@pytest.mark.parametrize("name,gen", [("philox4x32_10", srng.SRNG_PHILOX4X32_10),
                                      ("philox4x32_10_keyed", srng.SRNG_PHILOX4X32_10_KEYED),
                                      ("threefry4x32_20", srng.SRNG_THREEFRY4X32_20),
                                      ("threefry4x64_20", srng.SRNG_THREEFRY4X64_20),
                                      ("tinymt32", srng.SRNG_TINYMT32)])
def test_other_generators(name, gen):
    c = FIX["cases"][name]
    h = srng.srng_create(gen, c["seed"], S)
    try:
        assert np.array_equal(_draw(h), np.array(c["u32"], dtype=np.uint32))
    finally:
        srng.srng_destroy(h)
