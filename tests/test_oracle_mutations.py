"""Mutation check of the oracle's pins: plausible mistakes planted in copies of
the oracle's C source (a wrong coefficient, a swapped operand, a dropped term,
a wrong constant, an off-by-one conversion) must each make at least one pin
fail.  Everything runs on the CPU; the regular oracle is untouched."""
import ctypes
import math
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from tests.conftest import find_libcurand

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "srng_oracle.c")

MUTATIONS = {
    "a12 coefficient": ("#define ORC_A12 1403580LL", "#define ORC_A12 1403581LL"),
    "a23 coefficient": ("#define ORC_A23 1370589LL", "#define ORC_A23 1370598LL"),
    "m2 modulus": ("#define ORC_M2 4294944443ULL", "#define ORC_M2 4294944437ULL"),
    "component 1 lag": ("(ORC_A12 * (int64_t)s[1] - ORC_A13 * (int64_t)s[0])",
                        "(ORC_A12 * (int64_t)s[2] - ORC_A13 * (int64_t)s[0])"),
    "component 2 sign": ("(ORC_A21 * (int64_t)s[5] - ORC_A23 * (int64_t)s[3])",
                         "(ORC_A21 * (int64_t)s[5] + ORC_A23 * (int64_t)s[3])"),
    "combination wrap": ("return (uint32_t)(p1 - p2 + (int64_t)ORC_M1);", "return (uint32_t)(p1 - p2 + (int64_t)ORC_M2);"),
    "output from old state": ("    s[0] = s[1]; s[1] = s[2]; s[2] = (uint32_t)p1;\n",
                              "    s[0] = s[1]; s[1] = s[2]; s[2] = (uint32_t)p1; p1 = s[1];\n"),
    "matrix entry": ("a[2 * 3 + 1] = (uint64_t)ORC_A12;", "a[2 * 3 + 1] = (uint64_t)ORC_A13;"),
    "jump exponent word": ("uint64_t word = bit < 64 ? e_lo : e_hi;", "uint64_t word = bit < 63 ? e_lo : e_hi;"),
    "jump squaring": ("mat_mul(base, base, m, base);", "mat_mul(base, r, m, base);"),
    "philox multiplier": ("#define ORC_PHILOX_M0 0xD2511F53U", "#define ORC_PHILOX_M0 0xD2511F55U"),
    "philox weyl": ("#define ORC_PHILOX_W1 0xBB67AE85U", "#define ORC_PHILOX_W1 0xBB67AE86U"),
    "philox word order": ("uint32_t y1 = lo1;", "uint32_t y1 = lo0;"),
    "philox key use": ("uint32_t y2 = hi0 ^ x3 ^ k1;", "uint32_t y2 = hi0 ^ x3 ^ k0;"),
    "philox rounds": ("for (int round = 0; round < 10; ++round) {", "for (int round = 0; round < 9; ++round) {"),
    "f32 shift": ("return ldexpf((float)(v >> 8), -24);", "return ldexpf((float)(v >> 9), -23);"),
    "f64 norm": ("const double norm = 1.0 / 4294967088.0;", "const double norm = 1.0 / 4294967087.0;"),
    "philox f64 offset": ("return ((double)w + 0.5) / 4294967296.0;", "return ((double)w + 1.0) / 4294967296.0;"),
    "pi threshold philox": ("return a * a + b * b < ((unsigned __int128)1 << 48);",
                            "return a * a + b * b < ((unsigned __int128)1 << 47);"),
    "pi radius mrg": ("unsigned __int128 a = z0, b = z1, r = ORC_M1 + 1;", "unsigned __int128 a = z0, b = z1, r = ORC_M1;"),
    "ln2 low part sign": ("k->ln2_lo = (float)(ln2 - hi);", "k->ln2_lo = (float)(hi - ln2);"),
    "atanh series term": ("k->inv_odd[j] = 1.0f / (float)(2 * j + 1);", "k->inv_odd[j] = 1.0f / (float)(2 * j + 3);"),
    "ln leading term": ("float ln_m = fmaf(2.0f * s, s2 * p, 2.0f * s);", "float ln_m = fmaf(2.0f * s, s2 * p, s);"),
    "taylor sign": ("k->sc[n] = (float)(((n / 2) % 2) ? -t : t);", "k->sc[n] = (float)((n % 2) ? -t : t);"),
    "quadrant order": ("else if (q % 4 == 1) { *sin_out = cs; *cos_out = -sn; }",
                       "else if (q % 4 == 1) { *sin_out = cs; *cos_out = sn; }"),
    "reflection": ("if (exchanged) r = 1.0f - r;", "if (exchanged) r = r - 0.5f;"),
    "threefry permutation": ("        v[1] = v[3];\n        v[3] = t;\n", "        (void)t;\n"),
    "threefry rounds": ("for (int d = 0; d < 20; ++d) {", "for (int d = 0; d < 3; ++d) {"),
    "threefry64 permutation": ("        uint64_t t = v[1];\n        v[1] = v[3];\n        v[3] = t;\n",
                               "        uint64_t t = v[1];\n        (void)t;\n"),
    "threefry64 rounds": ("    for (int d = 0; d < 20; ++d) {\n        for (int pair = 0; pair < 2; ++pair) {\n            uint64_t",
                          "    for (int d = 0; d < 3; ++d) {\n        for (int pair = 0; pair < 2; ++pair) {\n            uint64_t"),
    "tinymt shift": ("    s[2] = x ^ (y << 10);", "    s[2] = x ^ (y << 11);"),
    "tinymt feedback": ("    x ^= x << 1;\n    uint32_t y", "    x ^= x << 2;\n    uint32_t y"),
    "tinymt mask": ("uint32_t x = (s[0] & ORC_TMT_MASK) ^ s[1] ^ s[2];", "uint32_t x = s[0] ^ s[1] ^ s[2];"),
    "tinymt horner order": ("    for (int i = 126; i >= 0; --i) {\n        oracle_tinymt32_next(acc",
                            "    for (int i = 0; i <= 126; ++i) {\n        oracle_tinymt32_next(acc"),
    "splitmix64 shift": ("z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBULL;"),
    "splitmix64 multiplier": ("0xBF58476D1CE4E5B9ULL", "0xBF58476D1CE4E5B7ULL"),
    "splitmix64 final shift": ("return z ^ (z >> 31);", "return z ^ (z >> 33);"),
    "tinymt tempering shift": ("uint32_t t = s[0] + (s[2] >> 8);", "uint32_t t = s[0] + (s[2] >> 9);"),
    "tinymt tempering word": ("uint32_t t = s[0] + (s[2] >> 8);", "uint32_t t = s[1] + (s[2] >> 8);"),
    "tinymt seeding shift": ("s[i % 4] ^= i + 1812433253U * (prev ^ (prev >> 30));",
                             "s[i % 4] ^= i + 1812433253U * (prev ^ (prev >> 27));"),
    "tinymt seeding multiplier": ("1812433253U", "1812433255U"),
    "threefry swapped mix pair": ("*b = orc_rotl32(*b, ORC_THREEFRY_ROT[d % 8][pair]) ^ *a;",
                                  "*b = orc_rotl32(*b, ORC_THREEFRY_ROT[d % 8][1 - pair]) ^ *a;"),
    "threefry rotation value": ("{10, 26}, {11, 21}", "{10, 25}, {11, 21}"),
    "threefry parity": ("#define ORC_THREEFRY_PARITY 0x1BD11BDAU", "#define ORC_THREEFRY_PARITY 0x1BD11BDBU"),
    "threefry injection count": ("            for (int i = 0; i < 4; ++i) v[i] += ks[(j + i) % 5];\n            v[3] += j;",
                                 "            for (int i = 0; i < 4; ++i) v[i] += ks[(j + i) % 5];\n            v[3] += 0;"),
    "threefry64 rotation value": ("{14, 16}, {52, 57}", "{14, 17}, {52, 57}"),
    "threefry64 parity": ("#define ORC_THREEFRY64_PARITY 0x1BD11BDAA9FC1A22ULL",
                          "#define ORC_THREEFRY64_PARITY 0x1BD11BDAA9FC1A23ULL"),
    "box-muller radius": ("float r = sqrtf(-2.0f * orc_ln(&k, 1.0f - in[2 * j]));",
                          "float r = sqrtf(-2.0f * orc_ln(&k, in[2 * j]));"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, name
    mutated = src.replace(old, new, 1)
    c = tmp_path / (name.replace(" ", "_") + ".c")
    c.write_text(mutated)
    so = tmp_path / (name.replace(" ", "_") + ".so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", str(c), "-o",
                    str(so), "-lm"], check=True)
    return str(so)


def _curand_outputs():
    path = find_libcurand()
    if path is None:
        return None
    lib = ctypes.CDLL(path)
    g = ctypes.c_void_p()
    lib.curandCreateGeneratorHost(ctypes.byref(g), 121)
    lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(0))
    buf = (ctypes.c_double * 64)()
    lib.curandGenerateUniformDouble(g, buf, ctypes.c_size_t(64))
    lib.curandDestroyGenerator(g)
    mrg = np.rint(np.frombuffer(buf, dtype=np.float64) * O.M1).astype(np.uint64)
    g = ctypes.c_void_p()
    lib.curandCreateGeneratorHost(ctypes.byref(g), 161)
    lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(0x0123456789ABCDEF))
    pb = (ctypes.c_uint32 * 64)()
    lib.curandGenerate(g, pb, ctypes.c_size_t(64))
    lib.curandDestroyGenerator(g)
    return mrg, np.frombuffer(pb, dtype=np.uint32).copy()


def _pymatpow(a, e, m):
    r = [[int(i == j) for j in range(3)] for i in range(3)]
    a = [[int(x) for x in row] for row in a]
    while e:
        if e & 1:
            r = [[sum(r[i][k] * a[k][j] for k in range(3)) % m for j in range(3)] for i in range(3)]
        a = [[sum(a[i][k] * a[k][j] for k in range(3)) % m for j in range(3)] for i in range(3)]
        e >>= 1
    return r


def _pins_fail(ref):
    """True if any pin (a subset of tests/test_oracle_pins.py) fails."""
    try:
        # third-party implementation (cuRAND host generators)
        if ref is not None:
            mrg, phx = ref
            starts = O.mrg_stream_starts([12345] * 6, 76, 0, 64)
            first = np.array([O.mrg_generate(st, 1)[0][0] for st in starts], dtype=np.uint64)
            if not np.array_equal(first, mrg):
                return True
            key = (0x89ABCDEF, 0x01234567)
            for s in range(16):
                if list(O.philox4x32_10([0, 0, s, 0], key)) != list(phx[4 * s: 4 * s + 4]):
                    return True
        # period 2^191: each component matrix has order m^3 - 1 (identity at the order)
        for comp, m in ((0, O.M1), (1, O.M2)):
            if not np.array_equal(O.mrg_matpow(comp, m**3 - 1), np.eye(3, dtype=np.uint64)):
                return True
        # 128-bit exponents (both words, bit 63 set) against Python big-int powers
        for comp, m in ((0, O.M1), (1, O.M2)):
            e = (1 << 63) | (1 << 64) | (1 << 100) | 12345
            if O.mrg_matpow(comp, e).tolist() != _pymatpow(O.mrg_matrix(comp).tolist(), e, m):
                return True
        # jump equals stepping
        s = [1, 2, 3, 4, 5, 6]
        _, stepped = O.mrg_generate(s, 1000)
        if list(O.mrg_jump(s, 1000)) != list(stepped):
            return True
        # step agrees with its matrix (unit states)
        a = O.mrg_matrix(0)
        _, st = O.mrg_step([1, 0, 0, 1, 2, 3])
        if [int(x) for x in st[:3]] != [int(a[i][0]) for i in range(3)]:
            return True
        # conversions against exact rationals
        for v in (0, 255, 256, 2**24, 2**31 + 5, 2**32 - 1):
            if Fraction(O.to_f32(v)) != Fraction(v >> 8, 1 << 24):
                return True
            if Fraction(O.philox_to_f64(v)) != Fraction(2 * v + 1, 1 << 33):
                return True
        norm = O.mrg_to_f64(1)
        if Fraction(norm) != Fraction(float(Fraction(1, O.M1 + 1))):
            return True
        # hit tests against exact geometry near the circle
        av = 11863283
        for b in range(av - 3, av + 4):
            if O.pi_hit_philox(av << 8, b << 8) != (av * av + b * b < 1 << 48):
                return True
        r = O.M1 + 1
        z0 = 3037000000
        z1 = math.isqrt(r * r - z0 * z0)
        for d in (-1, 0, 1, 2):
            if O.pi_hit_mrg(z0, z1 + d) != (z0 * z0 + (z1 + d) ** 2 < r * r):
                return True
        # output range
        z, _ = O.mrg_generate([7, 8, 9, 10, 11, 12], 2000)
        if z.min() < 1 or int(z.max()) > O.M1:
            return True
        # variates: float64 libm on a strided subset of the FP32 uniforms
        u = np.arange(1, 1 << 24, 251, dtype=np.float64) * 2.0**-24
        sp = lambda r: np.spacing(np.abs(r).astype(np.float32)).astype(np.float64)
        ref = -np.log1p(-u)
        if np.any(np.abs(O.transform(O.DIST_EXPONENTIAL, u.astype(np.float32)) - ref) > 2 * sp(ref)):
            return True
        s, c = O.sincos_2pi_array(u.astype(np.float32))
        t = 2 * np.pi * u
        if np.any(np.abs(s - np.sin(t)) > 2 * sp(np.sin(t)) + 1e-12) or \
                np.any(np.abs(c - np.cos(t)) > 2 * sp(np.cos(t)) + 1e-12):
            return True
        w = u[: (u.size // 2) * 2].astype(np.float32)
        g = O.transform(O.DIST_NORMAL, w).astype(np.float64)
        r = np.sqrt(-2 * np.log1p(-w[0::2].astype(np.float64)))
        if np.any(np.abs(g[0::2] - r * np.cos(2 * np.pi * w[1::2].astype(np.float64))) > 4 * sp(r) + 1e-12):
            return True
        # Threefry: every counter bit diffuses into every output bit
        rng = np.random.default_rng(7)
        flips = np.zeros((128, 128))
        for _ in range(48):
            ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
            key = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
            base = np.unpackbits(O.threefry4x32_20(ctr, key).view(np.uint8))
            for b in range(128):
                c2 = ctr.copy()
                c2[b // 32] ^= np.uint32(1 << (b % 32))
                flips[b] += np.unpackbits(O.threefry4x32_20(c2, key).view(np.uint8)) != base
        if np.abs(flips / 48 - 0.5).max() > 0.33:
            return True
        flips = np.zeros((256, 256))
        for _ in range(32):
            ctr = rng.integers(0, 2**63, 4, dtype=np.uint64)
            key = rng.integers(0, 2**63, 4, dtype=np.uint64)
            base = np.unpackbits(O.threefry4x64_20(ctr, key).view(np.uint8))
            for b in range(256):
                c2 = ctr.copy()
                c2[b // 64] ^= np.uint64(1 << (b % 64))
                flips[b] += np.unpackbits(O.threefry4x64_20(c2, key).view(np.uint8)) != base
        if np.abs(flips / 32 - 0.5).max() > 0.38:
            return True
        # SplitMix64 against pybind11's mix64 (when installed)
        from tests.independent import pybind11_mix64
        mix = pybind11_mix64()
        if mix is not None:
            gamma = 0x9E3779B97F4A7C15
            for seed in (0, 0x5EED5EED5EED5EED, 2**64 - 1):
                if O.splitmix64(seed, 4) != [mix((seed + (k + 1) * gamma) % 2**64) for k in range(4)]:
                    return True
        # Threefry: the inverse rounds take output blocks back to their counters
        from tests.test_oracle_threefry import _threefry_inverse
        rr = np.random.default_rng(3)
        for bits, f in ((32, O.threefry4x32_20), (64, O.threefry4x64_20)):
            for _ in range(8):
                ctr = [int(x) for x in rr.integers(0, 2**31, 4)]
                key = [int(x) for x in rr.integers(0, 2**31, 4)]
                if _threefry_inverse(f(ctr, key), key, bits) != ctr:
                    return True
        # TinyMT32: seeding through numpy's MT19937 mixer; tempering structure
        from tests.test_oracle_tinymt import _seed_from_mt19937_mixer
        dflt = (0x8F7011EE, 0xFC78FF1F, 0x3793FDFF)
        for seed in (1, 12345, 0xFFFFFFFF):
            if not np.array_equal(O.tinymt32_init(seed, dflt), _seed_from_mt19937_mixer(seed, dflt)):
                return True
        for st in ([5, 6, 7 << 9, 8], [0xFFFFFFFF, 3, 0x12345678, 0x9ABCDEF0]):
            t = (st[0] + (st[2] >> 8)) & 0xFFFFFFFF
            if O.tinymt32_temper(st, dflt[2]) != st[3] ^ t ^ (dflt[2] if t & 1 else 0):
                return True
        # TinyMT32: the authors' default parameter set has period 2^127 - 1
        # under the step; jumps equal stepping
        if not O.tinymt32_max_period(0x8F7011EE, 0xFC78FF1F):
            return True
        t0 = O.tinymt32_init(7, (0x8F7011EE, 0xFC78FF1F, 0x3793FDFF))
        t = t0.copy()
        for _ in range(300):
            t = O.tinymt32_next(t, 0x8F7011EE, 0xFC78FF1F)
        if not np.array_equal(O.tinymt32_jump(t0, 0x8F7011EE, 0xFC78FF1F, 300), t):
            return True
        return False
    except Exception:
        return True


def test_unmutated_oracle_passes_the_same_checks():
    O.use_library(None)
    assert not _pins_fail(_curand_outputs())


def test_every_planted_mistake_is_caught(tmp_path):
    ref = _curand_outputs()
    if ref is None:
        pytest.skip("libcurand not found")
    missed = []
    try:
        for name, (old, new) in MUTATIONS.items():
            O.use_library(_build(tmp_path, name, old, new))
            if not _pins_fail(ref):
                missed.append(name)
    finally:
        O.use_library(None)
    assert not missed, missed
