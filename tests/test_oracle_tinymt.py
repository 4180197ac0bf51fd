"""Pins of the oracle's TinyMT32 (Sec. 4.2: parameterised statuses shared by
the threads of a block, sequence splitting between the threads).

- The step: under it, the authors' default parameter set of TinyMT32
  (mat1 = 0x8f7011ee, mat2 = 0xfc78ff1f, Saito & Matsumoto 2011) has the
  maximal period 2^127 - 1 -- a property a wrong shift, mask or feedback
  destroys with probability about 126/127 -- checked with sympy's GF(2)
  arithmetic (an independent implementation), not the oracle's own.
- The characteristic polynomial annihilates every state bit's sequence.
- Jumps equal brute-force stepping, compose additively, and T^(2^127 - 1)
  is the identity.
- Parameter search: every set found has period 2^127 - 1 (sympy).
- Seeding: its mixing function x -> 1812433253 (x ^ (x >> 30)) is the MT19937
  initialisation's, taken here from numpy's MT19937 (an independent
  implementation run as a library); the seeding rebuilt from it (seven
  xor-mixing passes over (seed, mat1, mat2, tmat), the all-zero guard, eight
  steps) equals the oracle's for many seeds and parameter sets.
- Tempering: structure only -- it is a function of (s0, s2, s3) that does not
  read s1, reduces to s3 when s0 = s2 = 0 and tmat = 0, adds s2 >> 8 to s0
  and xors tmat exactly when that sum is odd; inverted here to recover s3.
  Its shift and the published form are restated from the publication, with
  no implementation here to compare outputs with, so the tempering stays
  parity unpinned beyond these properties."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.independent import mt19937_init_mix

DEFAULT = (0x8F7011EE, 0xFC78FF1F, 0x3793FDFF)


def _sympy_poly(coeffs):
    sympy = pytest.importorskip("sympy")
    x = sympy.Symbol("x")
    return sympy.Poly(sum(sympy.Integer(c) * x**i for i, c in enumerate(coeffs) if c), x, modulus=2), x


def _primitive_127(coeffs):
    """Degree 127, irreducible over GF(2) (hence primitive: 2^127 - 1 is prime),
    decided by sympy."""
    sympy = pytest.importorskip("sympy")
    p, x = _sympy_poly(coeffs)
    if p.degree() != 127 or not p.is_irreducible:
        return False
    # x^(2^127 - 1) = 1 mod p, by sympy's own modular powering
    r = sympy.Poly(1, x, modulus=2)
    base = sympy.Poly(x, x, modulus=2)
    e = 2**127 - 1
    while e:
        if e & 1:
            r = (r * base).rem(p)
        base = (base * base).rem(p)
        e >>= 1
    return r == sympy.Poly(1, x, modulus=2)


def test_default_parameter_set_has_maximal_period():
    p = O.tinymt32_charpoly(DEFAULT[0], DEFAULT[1])
    assert len(p) == 128 and _primitive_127(p)
    assert O.tinymt32_max_period(DEFAULT[0], DEFAULT[1])


def test_charpoly_annihilates_every_state_bit():
    p = O.tinymt32_charpoly(DEFAULT[0], DEFAULT[1])
    s = O.tinymt32_init(12345, DEFAULT)
    seq = []
    for _ in range(400):
        s = O.tinymt32_next(s, DEFAULT[0], DEFAULT[1])
        seq.append(s.copy())
    seq = np.array(seq, dtype=np.uint64)
    bits = np.stack([(seq[:, w] >> b) & 1 for w in range(4) for b in range(32) if not (w == 0 and b == 31)])
    idx = [i for i, c in enumerate(p) if c]
    for n in range(0, 400 - 128, 17):
        acc = np.zeros(bits.shape[0], dtype=np.uint64)
        for i in idx:
            acc ^= bits[:, n + i]
        assert not acc.any()


@pytest.mark.parametrize("J", [1, 2, 3, 127, 1000, 12345, 65543])
def test_jump_equals_stepping(J):
    s0 = O.tinymt32_init(7, DEFAULT)
    s = s0.copy()
    for _ in range(J):
        s = O.tinymt32_next(s, DEFAULT[0], DEFAULT[1])
    assert np.array_equal(O.tinymt32_jump(s0, DEFAULT[0], DEFAULT[1], J), s)


def test_jumps_compose_and_the_period_closes():
    s0 = O.tinymt32_init(99, DEFAULT)
    a, b = 2**100 + 12345, 2**64 * 7 + 3
    ab = O.tinymt32_jump(O.tinymt32_jump(s0, DEFAULT[0], DEFAULT[1], a), DEFAULT[0], DEFAULT[1], b)
    assert np.array_equal(ab, O.tinymt32_jump(s0, DEFAULT[0], DEFAULT[1], a + b))
    assert np.array_equal(O.tinymt32_jump(s0, DEFAULT[0], DEFAULT[1], 2**127 - 1), s0)
    assert not np.array_equal(O.tinymt32_jump(s0, DEFAULT[0], DEFAULT[1], 2**126), s0)


def test_found_parameter_sets_have_maximal_period():
    prm = O.tinymt32_find_params(0x5EED, 4)
    assert len({tuple(r) for r in prm}) == 4
    for mat1, mat2, _ in prm:
        assert _primitive_127(O.tinymt32_charpoly(int(mat1), int(mat2)))
    assert np.array_equal(prm, O.tinymt32_find_params(0x5EED, 4))     # deterministic
    assert not O.tinymt32_max_period(0, 0)


def test_bulk_stream_starts_equal_one_by_one():
    prm = O.tinymt32_find_params(5, 3)
    bulk = O.tinymt32_stream_starts(77, prm, 4, 10)
    for i in range(10):
        assert np.array_equal(bulk[i], O.tinymt32_stream_start(77, prm[i // 4], i % 4)), i


def test_stream_starts_are_substreams_2_64_apart():
    prm = O.tinymt32_find_params(3, 2)
    st = O.tinymt32_stream_starts(1, prm, 3, 6)
    for g in range(2):
        p = prm[g]
        base = O.tinymt32_init(1, p)
        assert np.array_equal(st[3 * g], base)
        assert np.array_equal(st[3 * g + 1], O.tinymt32_jump(base, int(p[0]), int(p[1]), 2**64))
        assert np.array_equal(st[3 * g + 2], O.tinymt32_jump(st[3 * g + 1], int(p[0]), int(p[1]), 2**64))


def test_generate_is_step_then_temper():
    s0 = O.tinymt32_init(5, DEFAULT)
    out, s_end = O.tinymt32_generate(s0, DEFAULT, 50)
    s = s0.copy()
    for k in range(50):
        s = O.tinymt32_next(s, DEFAULT[0], DEFAULT[1])
        assert int(out[k]) == O.tinymt32_temper(s, DEFAULT[2])
    assert np.array_equal(s, s_end)
    f, _ = O.tinymt32_generate(s0, DEFAULT, 50, O.OUT_F32)
    assert np.array_equal(f, (out >> 8).astype(np.float32) * np.float32(2.0**-24))


def test_output_bytes_uniform_and_streams_distinct():
    prm = O.tinymt32_find_params(11, 2)
    st = O.tinymt32_stream_starts(1, prm, 2, 4)
    out, _ = O.tinymt32_bulk(st, prm, 2, 1 << 16)
    counts = np.bincount(out.view(np.uint8).ravel(), minlength=256)
    e = out.size * 4 / 256
    assert ((counts - e) ** 2 / e).sum() < 400
    rows = {bytes(r[:64].tobytes()) for r in out}
    assert len(rows) == 4


def _seed_from_mt19937_mixer(seed32, prm):
    """TinyMT32 seeding with its multiply-xorshift taken from numpy's MT19937."""
    s = [seed32 & 0xFFFFFFFF, int(prm[0]), int(prm[1]), int(prm[2])]
    for i in range(1, 8):
        s[i % 4] ^= (i + mt19937_init_mix(s[(i - 1) % 4])) & 0xFFFFFFFF
    if (s[0] & 0x7FFFFFFF) == 0 and s[1] == s[2] == s[3] == 0:
        s = [ord("T"), ord("I"), ord("N"), ord("Y")]
    st = np.array(s, dtype=np.uint32)
    for _ in range(8):
        st = O.tinymt32_next(st, int(prm[0]), int(prm[1]))
    return st


def test_seeding_uses_the_mt19937_initialisation_mixer():
    rng = np.random.default_rng(42)
    sets = [DEFAULT] + [tuple(int(x) for x in r) for r in O.tinymt32_find_params(0x5EED, 3)]
    seeds = [0, 1, 12345, 0xFFFFFFFF, 0x80000000] + [int(x) for x in rng.integers(0, 2**32, 40)]
    for prm in sets:
        for seed in seeds:
            assert np.array_equal(O.tinymt32_init(seed, prm), _seed_from_mt19937_mixer(seed, prm)), (prm, seed)


def test_tempering_structure_and_inverse():
    rng = np.random.default_rng(7)
    tmat = DEFAULT[2]
    for _ in range(2000):
        s = [int(x) for x in rng.integers(0, 2**32, 4)]
        v = O.tinymt32_temper(s, tmat)
        # s1 is not read
        s_other = list(s)
        s_other[1] ^= 0xDEADBEEF
        assert O.tinymt32_temper(s_other, tmat) == v
        # recover s3 from the output: t = s0 + (s2 >> 8); v = s3 ^ t ^ (tmat if t odd)
        t = (s[0] + (s[2] >> 8)) & 0xFFFFFFFF
        assert v ^ t ^ (tmat if t & 1 else 0) == s[3]
        # tmat enters exactly when t is odd
        assert (O.tinymt32_temper(s, 0) ^ v) == (tmat if t & 1 else 0)
    for s3 in (0, 1, 0x12345678, 0xFFFFFFFF):
        assert O.tinymt32_temper([0, 77, 0, s3], 0) == s3
    # the shift of s2: bit k of s2 reaches bit k - 8 of t
    for k in range(8, 32):
        assert O.tinymt32_temper([0, 0, 1 << k, 0], 0) == 1 << (k - 8)
    for k in range(8):
        assert O.tinymt32_temper([0, 0, 1 << k, 0], 0) == 0
