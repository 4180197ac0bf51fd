// Host-side exact arithmetic: MRG32k3a jump matrices and the seed expansion.
//
// Jump-ahead (paper Sec. 2.3, sequence splitting; Sec. 4.1 gives the 2^127 /
// 2^76 stream and substream spacing of MRG32k3a): moving a state n draws
// forward is a product with the n-th power of each component's 3x3 transition
// matrix modulo its prime.  Powers are formed here, once, by
// square-and-multiply on exact 64-bit products; the device only applies them.
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "internal.h"

namespace srng_impl {

namespace {

// Transition matrices acting on (x[n-3], x[n-2], x[n-1]):
//   component 1: x[n] = 1403580 x[n-2] - 810728 x[n-3]  (mod m1)
//   component 2: x[n] = 527612 x[n-1] - 1370589 x[n-3]  (mod m2)
MatPair base_matrix()
{
    MatPair p;
    memset(&p, 0, sizeof p);
    uint32_t *a = p.a, *b = p.a + 9;
    a[1] = 1; a[5] = 1; a[6] = (uint32_t)(kM1 - 810728u); a[7] = 1403580u;
    b[1] = 1; b[5] = 1; b[6] = (uint32_t)(kM2 - 1370589u); b[8] = 527612u;
    return p;
}

void mul3(const uint32_t *x, const uint32_t *y, uint64_t m, uint32_t *out)
{
    uint32_t t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            uint64_t acc = 0;
            for (int k = 0; k < 3; ++k) acc += ((uint64_t)x[3 * i + k] * y[3 * k + j]) % m;
            t[3 * i + j] = (uint32_t)(acc % m);
        }
    memcpy(out, t, sizeof t);
}

std::mutex g_pow2_mu;
std::vector<MatPair> g_pow2;  // g_pow2[k] = A^(2^k)

}  // namespace

MatPair mat_identity()
{
    MatPair p;
    memset(&p, 0, sizeof p);
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < 3; ++i) p.a[9 * c + 4 * i] = 1;
    return p;
}

MatPair mat_mul(const MatPair &x, const MatPair &y)
{
    MatPair r;
    mul3(x.a, y.a, kM1, r.a);
    mul3(x.a + 9, y.a + 9, kM2, r.a + 9);
    return r;
}

MatPair mat_pow2(int k)
{
    std::lock_guard<std::mutex> lk(g_pow2_mu);
    if (g_pow2.empty()) g_pow2.push_back(base_matrix());
    while ((int)g_pow2.size() <= k) {
        const MatPair &last = g_pow2.back();
        g_pow2.push_back(mat_mul(last, last));
    }
    return g_pow2[k];
}

MatPair mat_pow_shifted(uint64_t n_hi, uint64_t n_lo, int shift)
{
    // (A^(2^shift))^n: multiply in A^(2^(shift + bit)) for every set bit of n.
    MatPair r = mat_identity();
    for (int bit = 0; bit < 128; ++bit) {
        uint64_t w = bit < 64 ? n_lo : n_hi;
        if ((w >> (bit & 63)) & 1) r = mat_mul(r, mat_pow2(shift + bit));
    }
    return r;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the state advances by the
// odd constant nearest 2^64 / golden ratio and each output is a bijective mix.
static uint64_t splitmix64(uint64_t &x)
{
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void seed_expand(uint64_t seed, uint32_t out[6])
{
    uint64_t x = seed;
    uint64_t r[6];
    for (int i = 0; i < 6; ++i) r[i] = splitmix64(x);
    for (int i = 0; i < 3; ++i) out[i] = (uint32_t)(r[i] % kM1);
    for (int i = 0; i < 3; ++i) out[3 + i] = (uint32_t)(r[3 + i] % kM2);
    if (!out[0] && !out[1] && !out[2]) out[0] = out[1] = out[2] = 12345u;
    if (!out[3] && !out[4] && !out[5]) out[3] = out[4] = out[5] = 12345u;
}

bool state_valid(const uint32_t s[6])
{
    for (int i = 0; i < 3; ++i)
        if (s[i] >= kM1) return false;
    for (int i = 3; i < 6; ++i)
        if (s[i] >= kM2) return false;
    if (!s[0] && !s[1] && !s[2]) return false;
    if (!s[3] && !s[4] && !s[5]) return false;
    return true;
}

}  // namespace srng_impl
