"""Helpers for the GPU parity tests: device buffers and numpy views."""
import numpy as np
import torch

import paper_1412_8266_gb300 as srng

TORCH_DTYPE = {srng.SRNG_OUT_U32: torch.int32, srng.SRNG_OUT_F32: torch.float32, srng.SRNG_OUT_F64: torch.float64}
NP_DTYPE = {srng.SRNG_OUT_U32: np.uint32, srng.SRNG_OUT_F32: np.float32, srng.SRNG_OUT_F64: np.float64}
BITS = {srng.SRNG_OUT_U32: np.uint32, srng.SRNG_OUT_F32: np.uint32, srng.SRNG_OUT_F64: np.uint64}


def dev():
    return torch.device("cuda", torch.cuda.current_device())


def empty(n, out_type, pad=0):
    """Device buffer of n elements (+pad in front, to test unaligned outputs)."""
    t = torch.empty(n + pad, dtype=TORCH_DTYPE[out_type], device=dev())
    return t, t[pad:]


def to_np(t, out_type):
    a = t.detach().cpu().numpy()
    return a.view(NP_DTYPE[out_type])


def bits(a, out_type):
    """Bit pattern view, so comparisons are bit-exact (also for NaN-free floats)."""
    return np.ascontiguousarray(a).view(BITS[out_type])


def assert_bitexact(got, ref, out_type, what=""):
    g = bits(np.asarray(got, dtype=NP_DTYPE[out_type]), out_type)
    r = bits(np.asarray(ref, dtype=NP_DTYPE[out_type]), out_type)
    assert g.shape == r.shape, (what, g.shape, r.shape)
    if not np.array_equal(g, r):
        bad = np.nonzero(g.ravel() != r.ravel())[0]
        raise AssertionError(f"{what}: {bad.size} of {g.size} differ; first at {bad[:8]}: "
                             f"got {g.ravel()[bad[:4]]} ref {r.ravel()[bad[:4]]}")


def key_of(seed):
    return (seed & 0xFFFFFFFF, seed >> 32)
