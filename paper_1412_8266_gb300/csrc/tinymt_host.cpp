// TinyMT32 host maths (paper Sec. 4.2): the step's characteristic polynomial,
// the maximal-period test, jump polynomials x^J mod p, the seeding of a
// parameter set, and the parameter search.  Polynomials over GF(2) are
// 128-bit words (bit i = coefficient of x^i); the characteristic polynomial
// has degree 127, every residue degree < 127.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "internal.h"

namespace srng_impl {

namespace {

void tmt_step(uint32_t s[4], uint32_t mat1, uint32_t mat2)
{
    uint32_t x = (s[0] & 0x7fffffffu) ^ s[1] ^ s[2];
    x ^= x << 1;
    const uint32_t y = s[3] ^ (s[3] >> 1) ^ x;
    const uint32_t m = 0u - (y & 1u);
    s[0] = s[1];
    s[1] = s[2] ^ (m & mat1);
    s[2] = x ^ (y << 10) ^ (m & mat2);
    s[3] = y;
}

// 256-bit words for Berlekamp-Massey (connection polynomials of degree < 256).
struct W256 {
    uint64_t w[4];
};

inline void shl_xor(W256 &c, const W256 &b, int m)  // c ^= b << m
{
    const int q = m >> 6, r = m & 63;
    for (int i = 3; i >= q; --i) {
        uint64_t v = b.w[i - q] << r;
        if (r && i - q - 1 >= 0) v |= b.w[i - q - 1] >> (64 - r);
        c.w[i] ^= v;
    }
}

inline int parity_and(const W256 &a, const W256 &b)
{
    uint64_t x = (a.w[0] & b.w[0]) ^ (a.w[1] & b.w[1]) ^ (a.w[2] & b.w[2]) ^ (a.w[3] & b.w[3]);
    return __builtin_parityll(x);
}

// The 16-bit spreading of a byte (bit i -> bit 2i), for squaring.
struct Spread {
    uint16_t t[256];
    Spread()
    {
        for (int v = 0; v < 256; ++v) {
            uint16_t s = 0;
            for (int i = 0; i < 8; ++i)
                if ((v >> i) & 1) s |= (uint16_t)(1u << (2 * i));
            t[v] = s;
        }
    }
};
const Spread g_spread;

// Reduction modulo p (degree 127): red[k] = x^(127 + k) mod p, k < 127.
struct Reducer {
    u128 red[127];
    explicit Reducer(u128 p)
    {
        const u128 low = p & ~((u128)1 << 127);  // x^127 = p - x^127 (mod p)
        red[0] = low;
        for (int k = 1; k < 127; ++k) {
            const u128 prev = red[k - 1];
            u128 v = prev << 1;
            if ((prev >> 126) & 1) v = (v & ~((u128)1 << 127)) ^ low;
            red[k] = v;
        }
    }
    // (hi:lo) -- a product of degree < 253 -- reduced to degree < 127
    u128 reduce(u128 lo, u128 hi) const
    {
        u128 r = lo & ~((u128)1 << 127);
        if ((lo >> 127) & 1) r ^= red[0];
        for (int half = 0; half < 2; ++half) {
            uint64_t w = (uint64_t)(hi >> (64 * half));
            while (w) {
                const int b = __builtin_ctzll(w);
                w &= w - 1;
                r ^= red[1 + 64 * half + b];  // bit 128 + 64 half + b = x^(127 + 1 + ...)
            }
        }
        return r;
    }
    u128 square(u128 a) const
    {
        u128 lo = 0, hi = 0;
        for (int byte = 0; byte < 16; ++byte) {
            const u128 s = (u128)g_spread.t[(uint8_t)(a >> (8 * byte))];
            if (byte < 8) lo |= s << (16 * byte);
            else hi |= s << (16 * (byte - 8));
        }
        return reduce(lo, hi);
    }
    u128 times_x(u128 a) const
    {
        u128 v = a << 1;
        if ((a >> 126) & 1) v = (v & ~((u128)1 << 127)) ^ red[0];
        return v;
    }
};

}  // namespace

void tmt_seed_state(uint32_t seed32, uint32_t mat1, uint32_t mat2, uint32_t tmat, uint32_t s[4])
{
    s[0] = seed32;
    s[1] = mat1;
    s[2] = mat2;
    s[3] = tmat;
    for (uint32_t i = 1; i < 8; ++i) {
        const uint32_t p = s[(i - 1) & 3];
        s[i & 3] ^= i + 1812433253u * (p ^ (p >> 30));
    }
    if ((s[0] & 0x7fffffffu) == 0 && s[1] == 0 && s[2] == 0 && s[3] == 0) {
        s[0] = 'T';
        s[1] = 'I';
        s[2] = 'N';
        s[3] = 'Y';
    }
    for (int i = 0; i < 8; ++i) tmt_step(s, mat1, mat2);
}

bool tmt_max_period(uint32_t mat1, uint32_t mat2, u128 *charpoly)
{
    // bit 0 of s2 along 254 steps; its minimal polynomial (Berlekamp-Massey)
    uint32_t s[4];
    tmt_seed_state(1, mat1, mat2, 0, s);
    uint8_t bits[254];
    for (int i = 0; i < 254; ++i) {
        tmt_step(s, mat1, mat2);
        bits[i] = s[2] & 1u;
    }
    W256 c = {{1, 0, 0, 0}}, b = {{1, 0, 0, 0}}, win = {{0, 0, 0, 0}};  // win bit i = bits[n - i]
    int L = 0, m = 1;
    for (int n = 0; n < 254; ++n) {
        const int d = bits[n] ^ parity_and(c, win);
        if (d) {
            const W256 t = c;
            shl_xor(c, b, m);
            if (2 * L <= n) {
                L = n + 1 - L;
                b = t;
                m = 1;
            } else {
                ++m;
            }
        } else {
            ++m;
        }
        // shift the window: bit i+1 <- bit i, bit 1 <- bits[n]
        for (int i = 3; i > 0; --i) win.w[i] = (win.w[i] << 1) | (win.w[i - 1] >> 63);
        win.w[0] = (win.w[0] << 1) | ((uint64_t)bits[n] << 1);
    }
    if (L != 127) return false;
    u128 p = 0;  // reciprocal: p_i = c_(127 - i)
    for (int i = 0; i <= 127; ++i)
        if ((c.w[i >> 6] >> (i & 63)) & 1) p |= (u128)1 << (127 - i);
    // no root in GF(2): p(0) = 1 and an odd number of terms
    const int terms = __builtin_popcountll((uint64_t)p) + __builtin_popcountll((uint64_t)(p >> 64));
    if (!(p & 1) || !(terms & 1)) return false;
    // x^(2^127) = x (mod p): with 127 prime, p is irreducible (and primitive)
    const Reducer rd(p);
    u128 r = 2;
    for (int i = 0; i < 127; ++i) r = rd.square(r);
    if (r != 2) return false;
    if (charpoly) *charpoly = p;
    return true;
}

u128 tmt_xpow(u128 p, uint64_t e_hi, uint64_t e_lo)
{
    const Reducer rd(p);
    u128 r = 1;
    bool started = false;
    for (int bit = 127; bit >= 0; --bit) {
        const uint64_t word = bit >= 64 ? e_hi : e_lo;
        const bool one = (word >> (bit & 63)) & 1;
        if (started) r = rd.square(r);
        if (one) {
            r = rd.times_x(r);
            started = true;
        }
    }
    return r;
}

u128 tmt_square_mod(u128 p, u128 a) { return Reducer(p).square(a); }

void tmt_find_params(uint64_t seed, uint32_t count, uint32_t *out, u128 *polys)
{
    // candidate k takes SplitMix64 outputs 2k and 2k+1 of the seed's sequence;
    // candidates are tested in parallel batches and kept in order
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    auto mix = [](uint64_t z) {
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    unsigned nt = std::thread::hardware_concurrency();
    nt = std::max(1u, std::min(nt, 64u));
    const uint64_t batch = 256ull * nt;
    uint32_t found = 0;
    std::vector<uint8_t> ok(batch);
    std::vector<u128> pp(batch);
    for (uint64_t k0 = 0; found < count; k0 += batch) {
        std::atomic<uint64_t> next{0};
        auto work = [&]() {
            for (uint64_t i; (i = next.fetch_add(1)) < batch;) {
                const uint64_t k = k0 + i;
                const uint64_t a = mix(seed + (2 * k + 1) * gamma);
                ok[i] = tmt_max_period((uint32_t)a, (uint32_t)(a >> 32), &pp[i]) ? 1 : 0;
            }
        };
        std::vector<std::thread> th;
        for (unsigned t = 1; t < nt; ++t) th.emplace_back(work);
        work();
        for (auto &t : th) t.join();
        for (uint64_t i = 0; i < batch && found < count; ++i) {
            if (!ok[i]) continue;
            const uint64_t k = k0 + i;
            const uint64_t a = mix(seed + (2 * k + 1) * gamma);
            const uint64_t b = mix(seed + (2 * k + 2) * gamma);
            out[3 * found] = (uint32_t)a;
            out[3 * found + 1] = (uint32_t)(a >> 32);
            out[3 * found + 2] = (uint32_t)b;
            if (polys) polys[found] = pp[i];
            ++found;
        }
    }
}

}  // namespace srng_impl
