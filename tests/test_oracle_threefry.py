"""Structure pins of the oracle's Threefry4x32-20 and Threefry4x64-20 (Sec. 4.3
names Threefry beside Philox).  Their rotation counts and key-schedule parity
constants come from Salmon et al. 2011 and no independent implementation is
available to compare with, so their values are parity unpinned; what is
pinned here holds for the construction whatever the constants: the stream
layout, diffusion of every counter and key bit into every output bit, uniform
bytes, distinct blocks for distinct counters (the block function is a
permutation), and -- the round structure -- an inverse written here from the
definition (undo the key injection, the word permutation and each MIX, round
by round, from the last) that takes every output block back to its counter,
which fails for a wrong rotation, a swapped MIX pair, a missing injection
count or a wrong parity constant in either the oracle or this inverse."""
import random

import numpy as np
import pytest

from oracle import oracle as O

# Rotation pairs and parity constants of the two Threefry forms (Salmon et al.
# 2011; the 64-bit ones are Threefish-256's), written out again for the inverse.
R32 = [(10, 26), (11, 21), (13, 27), (23, 5), (6, 20), (17, 11), (25, 10), (18, 20)]
R64 = [(14, 16), (52, 57), (23, 40), (5, 37), (25, 33), (46, 12), (58, 22), (32, 32)]
PARITY = {32: 0x1BD11BDA, 64: 0x1BD11BDAA9FC1A22}


def _threefry_inverse(out, key, bits):
    """Counter of the Threefry-4xbits-20 block `out` under `key`, by running the
    twenty rounds backwards: subtract the injected subkey (and its count), undo
    the (0, 3, 2, 1) permutation, then each MIX (b = rotr(b ^ a), a -= b)."""
    mask = (1 << bits) - 1
    rot = R32 if bits == 32 else R64
    ks = [int(k) for k in key]
    par = PARITY[bits]
    for k in ks:
        par ^= k
    ks.append(par)
    v = [int(x) for x in out]
    for d in range(19, -1, -1):
        if d % 4 == 3:
            j = (d + 1) // 4
            v = [(v[i] - ks[(j + i) % 5]) & mask for i in range(4)]
            v[3] = (v[3] - j) & mask
        v[1], v[3] = v[3], v[1]
        for pair in (0, 1):
            a, b = v[2 * pair], v[2 * pair + 1]
            r = rot[d % 8][pair]
            b ^= a
            b = ((b >> r) | (b << (bits - r))) & mask
            a = (a - b) & mask
            v[2 * pair], v[2 * pair + 1] = a, b
    return [(v[i] - ks[i]) & mask for i in range(4)]


@pytest.mark.parametrize("bits", [32, 64])
def test_inverse_rounds_recover_the_counter(bits):
    rng = random.Random(bits)
    f = O.threefry4x32_20 if bits == 32 else O.threefry4x64_20
    for t in range(300):
        ctr = [rng.getrandbits(bits) for _ in range(4)]
        key = [rng.getrandbits(bits) for _ in range(4)]
        if t < 4:  # edge blocks: zero and all-ones counters and keys
            ctr = [0 if t % 2 == 0 else (1 << bits) - 1] * 4
            key = [0 if t < 2 else (1 << bits) - 1] * 4
        assert _threefry_inverse(f(ctr, key), key, bits) == ctr


def test_word_layout():
    """Word p of stream s = word p mod 4 of the block with counter
    (p/4 low, p/4 high, 0, 0) under key (s low, s high, seed low, seed high)."""
    seed, s = 0x0123456789ABCDEF, (7 << 40) | 12345
    key = [s & 0xFFFFFFFF, s >> 32, seed & 0xFFFFFFFF, seed >> 32]
    for p in (0, 1, 2, 3, 4, 7, 2**34 + 5, 2**64 - 1):
        q = p // 4
        blk = O.threefry4x32_20([q & 0xFFFFFFFF, q >> 32, 0, 0], key)
        assert O.threefry_word(seed, s, p) == int(blk[p % 4])
    got = O.threefry_generate(seed, s, 5, 11)
    assert [int(x) for x in got] == [O.threefry_word(seed, s, 5 + k) for k in range(11)]


def test_generate_conversions_follow_the_words():
    seed, s = 99, 3
    w = O.threefry_generate(seed, s, 0, 64)
    f = O.threefry_generate(seed, s, 0, 64, O.OUT_F32)
    d = O.threefry_generate(seed, s, 0, 64, O.OUT_F64)
    assert np.array_equal(f, (w >> 8).astype(np.float32) * np.float32(2.0**-24))
    assert np.array_equal(d, (2.0 * w.astype(np.float64) + 1) * 2.0**-33)


def test_bulk_matches_per_stream_and_advances():
    out, pos = O.threefry_bulk(5, 10, [0, 3, 7], 9, O.OUT_U32)
    for i, p in enumerate([0, 3, 7]):
        assert np.array_equal(out[i], O.threefry_generate(5, 10 + i, p, 9))
    assert list(pos) == [9, 12, 16]


@pytest.mark.parametrize("which", ["counter", "key"])
def test_avalanche(which):
    """Flipping any one of the 128 counter (or key) bits flips each of the 128
    output bits with probability 1/2: over 200 random inputs, every
    (input bit, output bit) frequency lies in 0.5 +- 0.16 (> 4.5 sigma)."""
    rng = np.random.default_rng(1 if which == "counter" else 2)
    trials = 200
    flips = np.zeros((128, 128))
    for _ in range(trials):
        ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        base = np.unpackbits(O.threefry4x32_20(ctr, key).view(np.uint8))
        for b in range(128):
            c2, k2 = ctr.copy(), key.copy()
            tgt = c2 if which == "counter" else k2
            tgt[b // 32] ^= np.uint32(1 << (b % 32))
            flips[b] += np.unpackbits(O.threefry4x32_20(c2, k2).view(np.uint8)) != base
    freq = flips / trials
    assert np.abs(freq - 0.5).max() < 0.16


def test_uniform_bytes_and_distinct_blocks():
    """2^18 words of one stream: byte frequencies pass a chi-square test
    (255 degrees of freedom, threshold far in the tail), and the 2^16 blocks
    (consecutive counters) are pairwise distinct."""
    w = O.threefry_generate(0xC0FFEE, 0, 0, 1 << 18)
    counts = np.bincount(w.view(np.uint8), minlength=256)
    e = w.size * 4 / 256
    chi2 = ((counts - e) ** 2 / e).sum()
    assert chi2 < 400
    blocks = w.view(np.dtype((np.void, 16)))
    assert np.unique(blocks).size == blocks.size


def test_streams_and_seeds_differ():
    a = O.threefry_generate(1, 0, 0, 16)
    assert not np.array_equal(a, O.threefry_generate(1, 1, 0, 16))
    assert not np.array_equal(a, O.threefry_generate(2, 0, 0, 16))
    assert not np.array_equal(a, O.threefry_generate(1, 1 << 32, 0, 16))
    assert not np.array_equal(a, O.threefry_generate(1 << 32, 0, 0, 16))


# ------------------------------------------------------------- Threefry4x64-20
def test_4x64_word_layout():
    """Draw p = 32-bit word p mod 8 of block p / 8 (the low, then the high half
    of each 64-bit word) under key (stream, seed, 0, 0), counter (p / 8, 0, 0, 0)."""
    seed, s = 0x0123456789ABCDEF, (7 << 40) | 12345
    for p in (0, 1, 2, 7, 8, 15, 2**35 + 3, 2**64 - 1):
        blk = O.threefry4x64_20([p // 8, 0, 0, 0], [s, seed, 0, 0])
        w = int(blk[(p % 8) // 2])
        assert O.threefry64_word(seed, s, p) == ((w >> 32) if p % 2 else (w & 0xFFFFFFFF))
    got = O.threefry64_generate(seed, s, 5, 19)
    assert [int(x) for x in got] == [O.threefry64_word(seed, s, 5 + k) for k in range(19)]


def test_4x64_avalanche():
    """Every one of the 256 counter and key bits flips each of the 256 output
    bits with probability 1/2 (64 random inputs; 0.5 +- 0.27, > 4.3 sigma)."""
    rng = np.random.default_rng(3)
    trials = 64
    flips = np.zeros((512, 256))
    for _ in range(trials):
        ctr = rng.integers(0, 2**63, 4, dtype=np.uint64) * 2 + 1
        key = rng.integers(0, 2**63, 4, dtype=np.uint64) * 2
        base = np.unpackbits(O.threefry4x64_20(ctr, key).view(np.uint8))
        for b in range(512):
            c2, k2 = ctr.copy(), key.copy()
            tgt, bit = (c2, b) if b < 256 else (k2, b - 256)
            tgt[bit // 64] ^= np.uint64(1 << (bit % 64))
            flips[b] += np.unpackbits(O.threefry4x64_20(c2, k2).view(np.uint8)) != base
    assert np.abs(flips / trials - 0.5).max() < 0.27


def test_4x64_uniform_bytes_distinct_blocks_and_keys():
    w = O.threefry64_generate(0xC0FFEE, 0, 0, 1 << 18)
    counts = np.bincount(w.view(np.uint8), minlength=256)
    e = w.size * 4 / 256
    assert ((counts - e) ** 2 / e).sum() < 400
    blocks = w.view(np.dtype((np.void, 32)))
    assert np.unique(blocks).size == blocks.size
    a = O.threefry64_generate(1, 0, 0, 16)
    for other in (O.threefry64_generate(1, 1, 0, 16), O.threefry64_generate(2, 0, 0, 16),
                  O.threefry_generate(1, 0, 0, 16)):
        assert not np.array_equal(a, other)
