/*
 * srng_device.cuh -- device-side draws for CUDA kernels (sm_103a).
 *
 * The paper's device layer (arXiv 1412.8266, Sec. 5.2) constructs a generator
 * object inside the kernel, which picks up the calling thread's stream, and
 * calls next() on it.  Here the stream set's device view (srng_dev_view,
 * filled by srng_get_device_view in srng.h) is passed explicitly instead of
 * through hidden globals, so kernels stay pure functions of
 * (set, stream, position):
 *
 *     __global__ void foo(float* out, srng_dev_view v) {
 *         uint64_t s = blockIdx.x * blockDim.x + threadIdx.x;
 *         srng::Mrg32k3a g(v, s);            // loads stream s's state
 *         out[s] = g.next_f32();             // the paper's Listing 1
 *     }
 *
 * All arithmetic is exact integer arithmetic: MRG32k3a products are formed
 * with 32x32->64-bit multiplies and reduced modulo m = 2^32 - c by folding
 * (2^32 = c mod m), Philox uses the 32x32->64-bit products of its round
 * function, and the floating-point outputs are assembled from integer bits
 * (no FP64 pipe, no rounding other than the defined one).
 *
 * This header holds no allocation and no host code; it is the device math of
 * the library's own kernels too.
 */
#ifndef SRNG_DEVICE_CUH
#define SRNG_DEVICE_CUH

#include <stdint.h>

#include <type_traits>
#include <utility>
#if __cplusplus >= 202002L
#include <concepts>
#endif

#include "srng.h"

namespace srng {

/* ---------------------------------------------------------- MRG32k3a maths */
namespace mrg {
/* Moduli and recurrence coefficients (L'Ecuyer 1999, the generator of the
 * paper's Sec. 4.1):  x1[n] = (a12 x1[n-2] - a13 x1[n-3]) mod m1,
 *                     x2[n] = (a21 x2[n-1] - a23 x2[n-3]) mod m2. */
constexpr uint32_t kM1 = 4294967087u;  /* 2^32 - 209   */
constexpr uint32_t kM2 = 4294944443u;  /* 2^32 - 22853 */
constexpr uint32_t kC1 = 209u;
constexpr uint32_t kC2 = 22853u;
constexpr uint32_t kA12 = 1403580u;
constexpr uint32_t kA13 = 810728u;
constexpr uint32_t kA21 = 527612u;
constexpr uint32_t kA23 = 1370589u;

/* One step.  s0..s2 = (x1[n-3], x1[n-2], x1[n-1]), s3..s5 likewise for x2.
 * Returns z = (x1[n] - x2[n]) mod m1 in [1, m1].
 *
 * The two products of each component are formed as one 64-bit sum t; the
 * reduction then uses 2^32 = c (mod 2^32 - c) with 32-bit operations only
 * (carries instead of wide multiplies keep the integer multiply pipe, the
 * bottleneck of this recurrence on sm_103a, for the four main products):
 *
 * Component 1: t = a12 s1 + a13 (m1 - s0) = a12 s1 - a13 s0 (mod m1),
 *   t < 2^21 2^32 + 2^20 2^32 < 2^54, so t = h 2^32 + l with h < 2^22.
 *   p = h c1 < 2^30.  u = p + l (mod 2^32); on a carry u < p < 2^30, and the
 *   carried 2^32 is c1 mod m1, so v = u + c1 < 2^30 + 209.  Without a carry
 *   v = u < 2^32.  One conditional subtraction of m1 leaves v in [0, m1).
 * Component 2: t < 2^20 2^32 + 2^21 2^32 < 2^54, h < 2^22, and h c2 < 2^37
 *   is formed as one 64-bit product q = qh 2^32 + ql with qh <= 22.
 *   u = ql + l (mod 2^32) carries into qh (qh <= 23).  w = qh c2 < 525619;
 *   v = u + w (mod 2^32); on a carry v < w, and v + c2 < 2^20.  One
 *   conditional subtraction of m2 leaves v in [0, m2).
 *   Its t is assembled from 32-bit low and high products with a carry chain
 *   (dot2 below), which moves work from the 32x32->64 multiply to the faster
 *   32-bit multiplies (measured: 4% more draws per second than 64-bit
 *   products for both components, identical results). */
__device__ __forceinline__ void dot2(uint32_t a, uint32_t x, uint32_t b, uint32_t y, uint32_t &h, uint32_t &l)
{
    /* (h, l) = a x + b y, each product as mul.lo / mul.hi, the sum by add-with-carry */
    asm("{\n\t"
        "mul.lo.u32 %1, %2, %3;\n\t"
        "mul.hi.u32 %0, %2, %3;\n\t"
        "mad.lo.cc.u32 %1, %4, %5, %1;\n\t"
        "madc.hi.u32 %0, %4, %5, %0;\n\t"
        "}"
        : "=r"(h), "=r"(l)
        : "r"(a), "r"(x), "r"(b), "r"(y));
}

__device__ __forceinline__ uint32_t step(uint32_t &s0, uint32_t &s1, uint32_t &s2, uint32_t &s3,
                                         uint32_t &s4, uint32_t &s5)
{
    const uint64_t t1 = (uint64_t)kA12 * s1 + (uint64_t)kA13 * (kM1 - s0);
    const uint32_t h1 = (uint32_t)(t1 >> 32), l1 = (uint32_t)t1;
    const uint32_t p1 = h1 * kC1;
    const uint32_t u1 = p1 + l1;
    uint32_t v1 = u1 + (u1 < p1 ? kC1 : 0u);
    v1 = min(v1, v1 - kM1);               /* v1 >= m1 ? v1 - m1 : v1 (unsigned wrap) */

    uint32_t h2, l2;
    dot2(kA21, s5, kA23, kM2 - s3, h2, l2);
    const uint64_t q = (uint64_t)h2 * kC2;
    const uint32_t ql = (uint32_t)q;
    const uint32_t u2 = ql + l2;
    const uint32_t qh = (uint32_t)(q >> 32) + (u2 < ql ? 1u : 0u);
    const uint32_t w = qh * kC2;
    uint32_t v2 = u2 + w;
    v2 = v2 + (v2 < w ? kC2 : 0u);
    v2 = min(v2, v2 - kM2);

    s0 = s1; s1 = s2; s2 = v1;
    s3 = s4; s4 = s5; s5 = v2;
    const uint32_t d = v1 - v2;
    return v1 > v2 ? d : d + kM1;
}

/* x mod (2^32 - c) for any 64-bit x, c < 2^15 (three folds and one
 * conditional subtraction; used by the jump-ahead products). */
__device__ __forceinline__ uint32_t reduce64(uint64_t x, uint32_t c, uint32_t m)
{
    x = (x >> 32) * c + (uint32_t)x;  /* < 2^47 + 2^32         */
    x = (x >> 32) * c + (uint32_t)x;  /* < 2^30 + 2^32         */
    x = (x >> 32) * c + (uint32_t)x;  /* < 2^32 (see step())   */
    uint32_t r = (uint32_t)x;
    return min(r, r - m);
}

/* a 64-bit x folded once by 2^32 = c (mod 2^32 - c): hi c + lo, the same
 * residue, below 2^47 + 2^32 for c < 2^15 */
__device__ __forceinline__ uint64_t fold64(uint64_t x, uint32_t c)
{
    return (uint64_t)(uint32_t)(x >> 32) * c + (uint32_t)x;
}

/* (a M0 + b M1 + d M2) mod (2^32 - c) for entries and arguments below 2^32:
 * each product folded once (< 2^48), the three summed (< 2^50), the sum folded
 * once more -- its high word is below 2^18, so the result is below 2^34 --
 * then by its high word (below 4) into 32 bits with one carry correction,
 * and one conditional subtraction.  Seven 32x32 -> 64-bit products per dot
 * product where reducing every product in full took fifteen. */
__device__ __forceinline__ uint32_t dot3(uint32_t M0, uint32_t a, uint32_t M1, uint32_t b, uint32_t M2, uint32_t d,
                                         uint32_t c, uint32_t m)
{
    const uint64_t s = fold64((uint64_t)M0 * a, c) + fold64((uint64_t)M1 * b, c) + fold64((uint64_t)M2 * d, c);
    const uint64_t g = fold64(s, c);                                   /* < 2^18 c + 2^32 < 2^34 */
    const uint32_t gh = (uint32_t)(g >> 32), gl = (uint32_t)g;        /* gh < 4                 */
    uint32_t r = gl + gh * c;
    r += r < gl ? c : 0u;  /* a carry out of 32 bits is 2^32 = c: then r < gh c < 2^17, r + c < 2^32 */
    return min(r, r - m);
}

/* (y0, y1, y2) <- M (y0, y1, y2) mod m for a row-major 3x3 matrix M with
 * entries below m (m = 2^32 - c). */
__device__ __forceinline__ void matvec(const uint32_t *M, uint32_t &y0, uint32_t &y1, uint32_t &y2,
                                       uint32_t c, uint32_t m)
{
    const uint32_t r0 = dot3(M[0], y0, M[1], y1, M[2], y2, c, m);
    const uint32_t r1 = dot3(M[3], y0, M[4], y1, M[5], y2, c, m);
    const uint32_t r2 = dot3(M[6], y0, M[7], y1, M[8], y2, c, m);
    y0 = r0; y1 = r1; y2 = r2;
}

/* Apply a pair of jump matrices (A1^d, A2^d), 18 words: 9 for m1 then 9 for m2. */
__device__ __forceinline__ void jump(const uint32_t *M18, uint32_t &s0, uint32_t &s1, uint32_t &s2,
                                     uint32_t &s3, uint32_t &s4, uint32_t &s5)
{
    matvec(M18, s0, s1, s2, kC1, kM1);
    matvec(M18 + 9, s3, s4, s5, kC2, kM2);
}

/* double nearest to z * norm, norm = 0x1.000000d00000bp-32 (the double nearest
 * 1/(m1+1)), built from integers, for z in [1, m1].  norm = M 2^-84 with
 * M = 2^52 + w, w = 0xd00000b.  With k = bitlength(z) and zn = z 2^(32-k) in
 * [2^31, 2^32), the exact product is zn M 2^(k-116) and zn M = zn 2^52 + E,
 * E = zn w < 2^60, lies in [2^83, 2^84 + 2^60).  Below 2^84 its top 53 bits are
 * m = zn 2^21 + (E >> 31) with the 31-bit remainder E mod 2^31; at or above
 * 2^84 (only when zn is within 208 of 2^32) one more bit is shifted out.  The
 * remainder is rounded to nearest, ties to even, a carry into bit 53 moving
 * the exponent through the addition, and the exponent field is k + 990 (or
 * k + 991).  Equal, bit for bit, to the IEEE product for every z (checked
 * exhaustively on the device against the FP64 multiply). */
__device__ __forceinline__ double to_f64(uint32_t z)
{
    const uint32_t lz = (uint32_t)__clz(z);
    const uint32_t zn = z << lz;
    /* E = zn w with w = 0xd00000b: E >> 31 and E mod 2^31 are the high word
     * and half the (even) low word of zn (2w), 2w < 2^32. */
    const uint32_t elo = zn * 0x1A000016u;
    const uint32_t ehi = __umulhi(zn, 0x1A000016u);
    if (zn >= 0xFFFFFF30u) {
        /* The only inputs whose product can reach 2^84 (zn within 208 of 2^32;
         * below that zn 2^21 + ehi < (2^32 - 208) 2^21 + 2w < 2^53): general
         * path with a variable final shift. */
        uint64_t m = ((uint64_t)zn << 21) + ehi;
        uint32_t e = 1021u - lz;
        if (m >> 53) {
            const uint32_t rem = (elo >> 1) | ((uint32_t)m << 31);
            m >>= 1;
            m += (rem > 0x80000000u || (rem == 0x80000000u && (m & 1u))) ? 1u : 0u;
            e += 1;
        } else {
            m += (elo + ((uint32_t)m & 1u) > 0x80000000u) ? 1u : 0u;
        }
        return __longlong_as_double((long long)(((uint64_t)e << 52) + m));
    }
    /* m = zn 2^21 + ehi < 2^53 as (hi, lo); the exponent field (1021 - lz,
     * plus 1 from m's 2^52 bit) is added into hi; rounding to nearest even:
     * remainder elo / 2 > 2^30, or = 2^30 with m odd, i.e. elo + (m & 1) > 2^31,
     * i.e. elo + 2^31 - 1 + (m & 1) carries out of 32 bits (elo is even and at
     * most 2^32 - 2, so the sum is below 2^33).  m & 1 = ehi & 1 (zn 2^21 is
     * even), so that carry is known first and enters the sum forming m; as
     * elo is even, elo + (m & 1) = elo | (ehi & 1). */
    uint32_t lo, hi;
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %2, 2147483647;\n\t"
        "addc.cc.u32 %0, %3, %4;\n\t"
        "addc.u32 %1, %5, %6;\n\t}"
        : "=r"(lo), "=r"(hi)
        : "r"(elo | (ehi & 1u)), "r"(zn << 21), "r"(ehi), "r"(zn >> 11), "r"((1021u - lz) << 20));
    return __hiloint2double((int)hi, (int)lo);
}

/* The same value through the FP64 multiply (IEEE round to nearest even). */
__device__ __forceinline__ double to_f64_dmul(uint32_t z)
{
    return __dmul_rn((double)z, 0x1.000000d00000bp-32);
}

/* The same value through one FP64 fused multiply-add and no conversion: the
 * double with high word 0x43300000 and low word z is 2^52 + z exactly, and
 * (2^52 + z) norm - 2^52 norm is z norm exactly (2^52 norm is a double), so the
 * FMA's single rounding gives RN(z norm), the definition. */
__device__ __forceinline__ double to_f64_fma(uint32_t z)
{
    constexpr double kNorm = 0x1.000000d00000bp-32;
    return __fma_rn(__hiloint2double(0x43300000, (int)z), kNorm, -0x1p52 * kNorm);
}
}  // namespace mrg

/* ------------------------------------------------------ Philox4x32-10 maths */
namespace philox {
/* Multipliers and key increments of Philox4x32 (Salmon et al. 2011, the
 * generator of the paper's Sec. 4.3). */
constexpr uint32_t kM0 = 0xD2511F53u;
constexpr uint32_t kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u;
constexpr uint32_t kW1 = 0xBB67AE85u;

/* Ten rounds on counter (c0..c3) with key (k0, k1), in place.  The 64-bit
 * products are taken as separate low and high halves (mul.lo / mul.hi), which
 * sm_103a issues at a higher rate than one 32x32->64 multiply. */
__device__ __forceinline__ void block(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3,
                                      uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = kM0 * c0, hi0 = __umulhi(kM0, c0);
        const uint32_t lo1 = kM1 * c2, hi1 = __umulhi(kM1, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c1 = lo1;
        c3 = lo0;
        c0 = n0;
        c2 = n2;
        k0 += kW0;
        k1 += kW1;
    }
}

/* (2w + 1) 2^-33 as a double, exact, built from 32-bit integer operations.
 * With l = clz(w) (32 for w = 0), v = 2w + 1 has bit length 33 - l, and
 * x = v 2^l has bit 32 set: its low 32 bits are (w 2^l) 2 + 2^l (the two
 * terms share no bit).  The double is 2^(-l-1) (x / 2^32): its 52 fraction
 * bits are those low 32 bits followed by zeros, and its exponent field is
 * 1022 - l.  Shifts by 32 give 0 (PTX shl), which makes w = 0 come out as
 * 2^-33. */
__device__ __forceinline__ double to_f64(uint32_t w)
{
    const uint32_t l = (uint32_t)__clz(w);
    uint32_t wn, bit;
    asm("shl.b32 %0, %2, %3;\n\tshl.b32 %1, 1, %3;" : "=r"(wn), "=r"(bit) : "r"(w), "r"(l));
    const uint32_t x = (wn << 1) + bit;
    const uint32_t hi = ((1022u - l) << 20) + (x >> 12);
    return __hiloint2double((int)hi, (int)(x << 20));
}
}  // namespace philox

namespace threefry {
/* Threefry-4x32 (Salmon et al. 2011; the paper's Sec. 4.3 names it beside
 * Philox): add / rotate / xor on four 32-bit words in the Threefish pattern.
 * Round r pairs the words as (0,1),(2,3) when r is even and (0,3),(2,1) when
 * it is odd; in each pair a += b, b = rotl(b, R) ^ a, with the rotation counts
 * R of round r mod 8 below.  The key schedule has the four key words and their
 * xor with kParity; subkey j (j = 0 first, then after every fourth round) adds
 * key words j..j+3 (mod 5) to the state and j to word 3.  Twenty rounds. */
constexpr uint32_t kParity = 0x1BD11BDAu;
__host__ __device__ constexpr int rot(int r, int half)
{
    return r == 0 ? (half ? 26 : 10) : r == 1 ? (half ? 21 : 11) : r == 2 ? (half ? 27 : 13)
         : r == 3 ? (half ? 5 : 23) : r == 4 ? (half ? 20 : 6) : r == 5 ? (half ? 11 : 17)
         : r == 6 ? (half ? 10 : 25) : (half ? 20 : 18);
}

__device__ __forceinline__ uint32_t rotl(uint32_t x, int r) { return __funnelshift_l(x, x, r); }

/* Twenty rounds on counter (c0..c3) with key (k0..k3), in place. */
__device__ __forceinline__ void block(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t k0,
                                      uint32_t k1, uint32_t k2, uint32_t k3)
{
    const uint32_t ks[5] = {k0, k1, k2, k3, kParity ^ k0 ^ k1 ^ k2 ^ k3};
    c0 += ks[0]; c1 += ks[1]; c2 += ks[2]; c3 += ks[3];
#pragma unroll
    for (int r = 0; r < 20; ++r) {
        if ((r & 1) == 0) {
            c0 += c1; c1 = rotl(c1, rot(r & 7, 0)) ^ c0;
            c2 += c3; c3 = rotl(c3, rot(r & 7, 1)) ^ c2;
        } else {
            c0 += c3; c3 = rotl(c3, rot(r & 7, 0)) ^ c0;
            c2 += c1; c1 = rotl(c1, rot(r & 7, 1)) ^ c2;
        }
        if ((r & 3) == 3) {
            const int j = (r + 1) >> 2;
            c0 += ks[j % 5]; c1 += ks[(j + 1) % 5]; c2 += ks[(j + 2) % 5]; c3 += ks[(j + 3) % 5] + (uint32_t)j;
        }
    }
}
}  // namespace threefry

namespace threefry64 {
/* Threefry-4x64 (Salmon et al. 2011): the same construction on four 64-bit
 * words (the Threefish-256 shape) with parity constant kParity64 and the
 * rotation pairs of rot64; twenty rounds.  64-bit adds and rotates run as
 * pairs of 32-bit operations on this GPU. */
constexpr uint64_t kParity64 = 0x1BD11BDAA9FC1A22ull;
__host__ __device__ constexpr int rot64(int r, int half)
{
    return r == 0 ? (half ? 16 : 14) : r == 1 ? (half ? 57 : 52) : r == 2 ? (half ? 40 : 23)
         : r == 3 ? (half ? 37 : 5) : r == 4 ? (half ? 33 : 25) : r == 5 ? (half ? 12 : 46)
         : r == 6 ? (half ? 22 : 58) : (half ? 32 : 32);
}
__device__ __forceinline__ uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

/* Twenty rounds on counter (c0..c3) with key (k0..k3), in place. */
__device__ __forceinline__ void block(uint64_t &c0, uint64_t &c1, uint64_t &c2, uint64_t &c3, uint64_t k0,
                                      uint64_t k1, uint64_t k2, uint64_t k3)
{
    const uint64_t ks[5] = {k0, k1, k2, k3, kParity64 ^ k0 ^ k1 ^ k2 ^ k3};
    c0 += ks[0]; c1 += ks[1]; c2 += ks[2]; c3 += ks[3];
#pragma unroll
    for (int r = 0; r < 20; ++r) {
        if ((r & 1) == 0) {
            c0 += c1; c1 = rotl64(c1, rot64(r & 7, 0)) ^ c0;
            c2 += c3; c3 = rotl64(c3, rot64(r & 7, 1)) ^ c2;
        } else {
            c0 += c3; c3 = rotl64(c3, rot64(r & 7, 0)) ^ c0;
            c2 += c1; c1 = rotl64(c1, rot64(r & 7, 1)) ^ c2;
        }
        if ((r & 3) == 3) {
            const int j = (r + 1) >> 2;
            c0 += ks[j % 5]; c1 += ks[(j + 1) % 5]; c2 += ks[(j + 2) % 5]; c3 += ks[(j + 3) % 5] + (uint64_t)j;
        }
    }
}

/* The eight 32-bit draws of block q of stream s under `seed`: key (s, seed, 0, 0),
 * counter (q, 0, 0, 0); the low then the high half of each 64-bit word. */
__device__ __forceinline__ void words(uint64_t q, uint64_t s, uint64_t seed, uint32_t *w)
{
    uint64_t c0 = q, c1 = 0, c2 = 0, c3 = 0;
    block(c0, c1, c2, c3, s, seed, 0, 0);
    w[0] = (uint32_t)c0; w[1] = (uint32_t)(c0 >> 32); w[2] = (uint32_t)c1; w[3] = (uint32_t)(c1 >> 32);
    w[4] = (uint32_t)c2; w[5] = (uint32_t)(c2 >> 32); w[6] = (uint32_t)c3; w[7] = (uint32_t)(c3 >> 32);
}
}  // namespace threefry64

namespace tinymt {
/* TinyMT32 (Saito & Matsumoto 2011; the paper's Sec. 4.2): one step of the
 * 127-bit GF(2)-linear state (bit 31 of s0 unused) with parameters
 * (mat1, mat2); the conditional feedback of y's low bit as a mask. */
__device__ __forceinline__ void step(uint32_t &s0, uint32_t &s1, uint32_t &s2, uint32_t &s3, uint32_t mat1,
                                     uint32_t mat2)
{
    uint32_t x = (s0 & 0x7fffffffu) ^ s1 ^ s2;
    x ^= x << 1;
    const uint32_t y = s3 ^ (s3 >> 1) ^ x;
    const uint32_t m = 0u - (y & 1u);
    s0 = s1;
    s1 = s2 ^ (m & mat1);
    s2 = x ^ (y << 10) ^ (m & mat2);
    s3 = y;
}

/* The output of a stepped state: t = s0 + (s2 >> 8), s3 ^ t, ^ tmat if t is odd. */
__device__ __forceinline__ uint32_t temper(uint32_t s0, uint32_t s2, uint32_t s3, uint32_t tmat)
{
    const uint32_t t = s0 + (s2 >> 8);
    return s3 ^ t ^ ((0u - (t & 1u)) & tmat);
}

/* s <- r(T) s by Horner's rule, r a polynomial of degree < 127 over GF(2)
 * (bit i of the 128-bit (r.x, r.y, r.z, r.w) = coefficient of x^i): with
 * r = x^J mod p, p the characteristic polynomial, this is J steps.  The state
 * must come from at least one step (the unused bit then lies in the image). */
__device__ __forceinline__ void horner_word(uint32_t word, int hi, uint32_t &a0, uint32_t &a1, uint32_t &a2,
                                            uint32_t &a3, uint32_t s0, uint32_t s1, uint32_t s2, uint32_t s3,
                                            uint32_t mat1, uint32_t mat2)
{
    for (int b = hi; b >= 0; --b) {
        step(a0, a1, a2, a3, mat1, mat2);
        const uint32_t m = 0u - ((word >> b) & 1u);
        a0 ^= m & s0; a1 ^= m & s1; a2 ^= m & s2; a3 ^= m & s3;
    }
}
__device__ __forceinline__ void jump(const uint4 r, uint32_t &s0, uint32_t &s1, uint32_t &s2, uint32_t &s3,
                                     uint32_t mat1, uint32_t mat2)
{
    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    horner_word(r.w, 30, a0, a1, a2, a3, s0, s1, s2, s3, mat1, mat2);
    horner_word(r.z, 31, a0, a1, a2, a3, s0, s1, s2, s3, mat1, mat2);
    horner_word(r.y, 31, a0, a1, a2, a3, s0, s1, s2, s3, mat1, mat2);
    horner_word(r.x, 31, a0, a1, a2, a3, s0, s1, s2, s3, mat1, mat2);
    s0 = a0; s1 = a1; s2 = a2; s3 = a3;
}
}  // namespace tinymt

/* (v >> 8) 2^-24 as a float, exact, without an integer-to-float conversion:
 * with a = v >> 8 = 2k + b, the bit pattern 0x3F800000 | k is 1 + k 2^-23;
 * adding -1 (b = 0) or -(1 - 2^-24) (b = 1, the float 0x3F7FFFFF) leaves
 * (2k + b) 2^-24, which has at most 24 significant bits, so the one rounded
 * addition is exact. */
__device__ __forceinline__ float to_f32(uint32_t v)
{
    const float one_k = __uint_as_float(0x3F800000u | (v >> 9));
    const float minus = __uint_as_float((v & 0x100u) ? 0xBF7FFFFFu : 0xBF800000u);
    return __fadd_rn(one_k, minus);
}

/* The same value as to_f32 through the integer-to-float conversion unit:
 * v >> 8 has at most 24 significant bits, so the conversion and the scaling
 * by 2^-24 are both exact.  Kernels whose integer pipes are the busy ones
 * (the counter-based rounds) take this form. */
__device__ __forceinline__ float to_f32_cvt(uint32_t v)
{
    return __fmul_rn(__uint2float_rn(v >> 8), 0x1p-24f);
}

/* ------------------------------------------------------- generator objects */

namespace mrg {
/* Jump-ahead by any distance inside a kernel: (A1^n, A2^n) applied by square
 * and multiply (at most 64 matrix squarings and 64 matrix-vector products per
 * component), for a stream handle that starts at an offset (Sec. 2.3: the
 * start of draw n of a stream is A^n y).  The host tables of srng_jump serve
 * the library's own kernels; this serves user kernels. */
__device__ __forceinline__ void matmul(const uint32_t *A, const uint32_t *B, uint32_t *C, uint32_t c, uint32_t m)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            C[3 * i + j] = dot3(A[3 * i], B[j], A[3 * i + 1], B[3 + j], A[3 * i + 2], B[6 + j], c, m);
        }
}

__device__ inline void skip(uint64_t n, uint32_t &s0, uint32_t &s1, uint32_t &s2, uint32_t &s3, uint32_t &s4,
                            uint32_t &s5)
{
    uint32_t p1[9] = {0, 1, 0, 0, 0, 1, kM1 - kA13, kA12, 0};  /* A1^(2^k) */
    uint32_t p2[9] = {0, 1, 0, 0, 0, 1, kM2 - kA23, 0, kA21};  /* A2^(2^k) */
    while (n) {
        if (n & 1) {
            matvec(p1, s0, s1, s2, kC1, kM1);
            matvec(p2, s3, s4, s5, kC2, kM2);
        }
        n >>= 1;
        if (n) {
            uint32_t t[9];
            matmul(p1, p1, t, kC1, kM1);
            for (int k = 0; k < 9; ++k) p1[k] = t[k];
            matmul(p2, p2, t, kC2, kM2);
            for (int k = 0; k < 9; ++k) p2[k] = t[k];
        }
    }
}
}  // namespace mrg (device jump-ahead)

/* MRG32k3a stream handle: the paper's device RNG object with next(). */
class Mrg32k3a {
  public:
    __device__ Mrg32k3a(const srng_dev_view &v, uint64_t stream)
    {
        const uint64_t n = v.n_streams;
        s0 = v.mrg_state[0 * n + stream]; s1 = v.mrg_state[1 * n + stream];
        s2 = v.mrg_state[2 * n + stream]; s3 = v.mrg_state[3 * n + stream];
        s4 = v.mrg_state[4 * n + stream]; s5 = v.mrg_state[5 * n + stream];
    }
    /* Stream `stream` of the view, `offset` draws after its current position. */
    __device__ Mrg32k3a(const srng_dev_view &v, uint64_t stream, uint64_t offset) : Mrg32k3a(v, stream)
    {
        skip(offset);
    }
    __device__ explicit Mrg32k3a(const uint32_t st[6])
        : s0(st[0]), s1(st[1]), s2(st[2]), s3(st[3]), s4(st[4]), s5(st[5]) {}

    __device__ __forceinline__ uint32_t next_u32() { return mrg::step(s0, s1, s2, s3, s4, s5); }
    __device__ __forceinline__ float next_f32() { return to_f32(next_u32()); }
    __device__ __forceinline__ double next_f64() { return mrg::to_f64(next_u32()); }
    /* The next four draws as one vector (x first). */
    __device__ __forceinline__ uint4 next4()
    {
        uint4 r;
        r.x = next_u32(); r.y = next_u32(); r.z = next_u32(); r.w = next_u32();
        return r;
    }
    /* Jump by a precomputed matrix pair (A1^d, A2^d) (srng_jump_matrix). */
    __device__ __forceinline__ void jump(const uint32_t *M18) { mrg::jump(M18, s0, s1, s2, s3, s4, s5); }
    /* Move n draws ahead (square and multiply on the device). */
    __device__ void skip(uint64_t n) { mrg::skip(n, s0, s1, s2, s3, s4, s5); }
    /* Write the current state back (so a later launch continues from here). */
    __device__ void store(const srng_dev_view &v, uint64_t stream) const
    {
        const uint64_t n = v.n_streams;
        v.mrg_state[0 * n + stream] = s0; v.mrg_state[1 * n + stream] = s1;
        v.mrg_state[2 * n + stream] = s2; v.mrg_state[3 * n + stream] = s3;
        v.mrg_state[4 * n + stream] = s4; v.mrg_state[5 * n + stream] = s5;
    }

    uint32_t s0, s1, s2, s3, s4, s5;
};

/* Philox4x32-10 stream handle: counter words 0-1 = block index; words 2-3 =
 * the stream and key = the set's seed, or -- keyed layout -- key = the stream
 * and words 2-3 = the seed. */
class Philox4x32_10 {
  public:
    /* `stream` is the slot in the set; the key / counter use its stream number
     * v.stream_base + stream. */
    __device__ Philox4x32_10(const srng_dev_view &v, uint64_t stream)
        : k0((v.flags & 1u) ? (uint32_t)(v.stream_base + stream) : v.key0),
          k1((v.flags & 1u) ? (uint32_t)((v.stream_base + stream) >> 32) : v.key1), stream_(stream),
          ctr_hi_((v.flags & 1u) ? ((uint64_t)v.key1 << 32 | v.key0) : v.stream_base + stream),
          pos_(v.philox_pos[stream]), bq_(~0ull) {}
    /* Stream `stream` of the view, `offset` draws after its current position. */
    __device__ Philox4x32_10(const srng_dev_view &v, uint64_t stream, uint64_t offset) : Philox4x32_10(v, stream)
    {
        pos_ += offset;
    }
    __device__ Philox4x32_10(uint32_t key0, uint32_t key1, uint64_t stream, uint64_t position)
        : k0(key0), k1(key1), stream_(stream), ctr_hi_(stream), pos_(position), bq_(~0ull) {}

    /* The four words of block q of this stream. */
    __device__ __forceinline__ uint4 block(uint64_t q) const
    {
        uint32_t c0 = (uint32_t)q, c1 = (uint32_t)(q >> 32);
        uint32_t c2 = (uint32_t)ctr_hi_, c3 = (uint32_t)(ctr_hi_ >> 32);
        philox::block(c0, c1, c2, c3, k0, k1);
        return make_uint4(c0, c1, c2, c3);
    }
    /* Draw pos: the block of the previous draw is kept, so four consecutive
     * draws cost one block. */
    __device__ __forceinline__ uint32_t next_u32()
    {
        const uint64_t q = pos_ >> 2;
        if (q != bq_) {
            b_ = block(q);
            bq_ = q;
        }
        const uint32_t j = (uint32_t)pos_ & 3u;
        ++pos_;
        return j == 0 ? b_.x : j == 1 ? b_.y : j == 2 ? b_.z : b_.w;
    }
    __device__ __forceinline__ float next_f32() { return to_f32(next_u32()); }
    __device__ __forceinline__ double next_f64() { return philox::to_f64(next_u32()); }
    /* The next four draws as one vector (x first). */
    __device__ __forceinline__ uint4 next4()
    {
        uint4 r;
        r.x = next_u32(); r.y = next_u32(); r.z = next_u32(); r.w = next_u32();
        return r;
    }
    __device__ void store(const srng_dev_view &v) const { v.philox_pos[stream_] = pos_; }
    __device__ uint64_t position() const { return pos_; }

    uint32_t k0, k1;
    uint64_t stream_, ctr_hi_, pos_;

  private:
    uint64_t bq_;  // block held in b_ (~0: none; block numbers are below 2^62)
    uint4 b_;
};

/* Threefry4x32-20 stream handle (the paper's per-thread key, Sec. 4.3):
 * key = (stream low, stream high, seed low, seed high), counter = (q low,
 * q high, 0, 0) for block q; word p mod 4 of block p / 4 is draw p.  Doubles
 * and singles as for Philox. */
class Threefry4x32_20 {
  public:
    /* `stream` is the slot in the set; the key uses its stream number
     * v.stream_base + stream and the set's seed words v.key0, v.key1. */
    __device__ Threefry4x32_20(const srng_dev_view &v, uint64_t stream)
        : k0((uint32_t)(v.stream_base + stream)), k1((uint32_t)((v.stream_base + stream) >> 32)), k2(v.key0),
          k3(v.key1), stream_(stream), pos_(v.philox_pos[stream]), bq_(~0ull) {}
    __device__ Threefry4x32_20(const srng_dev_view &v, uint64_t stream, uint64_t offset) : Threefry4x32_20(v, stream)
    {
        pos_ += offset;
    }
    __device__ Threefry4x32_20(uint64_t seed, uint64_t stream, uint64_t position)
        : k0((uint32_t)stream), k1((uint32_t)(stream >> 32)), k2((uint32_t)seed), k3((uint32_t)(seed >> 32)),
          stream_(stream), pos_(position), bq_(~0ull) {}

    __device__ __forceinline__ uint4 block(uint64_t q) const
    {
        uint32_t c0 = (uint32_t)q, c1 = (uint32_t)(q >> 32), c2 = 0, c3 = 0;
        threefry::block(c0, c1, c2, c3, k0, k1, k2, k3);
        return make_uint4(c0, c1, c2, c3);
    }
    __device__ __forceinline__ uint32_t next_u32()
    {
        const uint64_t q = pos_ >> 2;
        if (q != bq_) {
            b_ = block(q);
            bq_ = q;
        }
        const uint32_t j = (uint32_t)pos_ & 3u;
        ++pos_;
        return j == 0 ? b_.x : j == 1 ? b_.y : j == 2 ? b_.z : b_.w;
    }
    __device__ __forceinline__ float next_f32() { return to_f32(next_u32()); }
    __device__ __forceinline__ double next_f64() { return philox::to_f64(next_u32()); }
    /* The next four draws as one vector (x first). */
    __device__ __forceinline__ uint4 next4()
    {
        uint4 r;
        r.x = next_u32(); r.y = next_u32(); r.z = next_u32(); r.w = next_u32();
        return r;
    }
    __device__ void store(const srng_dev_view &v) const { v.philox_pos[stream_] = pos_; }
    __device__ uint64_t position() const { return pos_; }

    uint32_t k0, k1, k2, k3;
    uint64_t stream_, pos_;

  private:
    uint64_t bq_;  // block held in b_ (~0: none)
    uint4 b_;
};

/* Threefry4x64-20 stream handle: key = (stream, seed, 0, 0), counter
 * (q, 0, 0, 0) for block q; draw p is 32-bit word p mod 8 of block p / 8. */
class Threefry4x64_20 {
  public:
    __device__ Threefry4x64_20(const srng_dev_view &v, uint64_t stream)
        : s_(v.stream_base + stream), seed_((uint64_t)v.key1 << 32 | v.key0), stream_(stream),
          pos_(v.philox_pos[stream]), bq_(~0ull) {}
    __device__ Threefry4x64_20(const srng_dev_view &v, uint64_t stream, uint64_t offset) : Threefry4x64_20(v, stream)
    {
        pos_ += offset;
    }
    __device__ Threefry4x64_20(uint64_t seed, uint64_t stream, uint64_t position)
        : s_(stream), seed_(seed), stream_(stream), pos_(position), bq_(~0ull) {}

    /* Eight consecutive draws cost one block (the last block is kept). */
    __device__ __forceinline__ uint32_t next_u32()
    {
        const uint64_t q = pos_ >> 3;
        if (q != bq_) {
            threefry64::words(q, s_, seed_, w_);
            bq_ = q;
        }
        const uint32_t j = (uint32_t)pos_ & 7u;
        ++pos_;
        uint32_t r = w_[0];
#pragma unroll
        for (int i = 1; i < 8; ++i) r = j == (uint32_t)i ? w_[i] : r;
        return r;
    }
    __device__ __forceinline__ float next_f32() { return to_f32(next_u32()); }
    __device__ __forceinline__ double next_f64() { return philox::to_f64(next_u32()); }
    /* The next four draws as one vector (x first). */
    __device__ __forceinline__ uint4 next4()
    {
        uint4 r;
        r.x = next_u32(); r.y = next_u32(); r.z = next_u32(); r.w = next_u32();
        return r;
    }
    __device__ void store(const srng_dev_view &v) const { v.philox_pos[stream_] = pos_; }
    __device__ uint64_t position() const { return pos_; }

    uint64_t s_, seed_, stream_, pos_;

  private:
    uint64_t bq_;  // block held in w_ (~0: none; block numbers are below 2^61)
    uint32_t w_[8];
};

/* TinyMT32 stream handle (the paper's Sec. 4.2 hybrid: the parameter set of
 * the stream's group, a CUDA block's threads, and the stream's own state). */
class TinyMT32 {
  public:
    __device__ TinyMT32(const srng_dev_view &v, uint64_t stream)
    {
        const uint64_t n = v.n_streams;
        s0 = v.tinymt_state[stream]; s1 = v.tinymt_state[n + stream];
        s2 = v.tinymt_state[2 * n + stream]; s3 = v.tinymt_state[3 * n + stream];
        const uint32_t *p = v.tinymt_params + 4 * (stream / v.tinymt_group_size);
        mat1 = p[0]; mat2 = p[1]; tmat = p[2];
    }
    __device__ __forceinline__ uint32_t next_u32()
    {
        tinymt::step(s0, s1, s2, s3, mat1, mat2);
        return tinymt::temper(s0, s2, s3, tmat);
    }
    __device__ __forceinline__ float next_f32() { return to_f32(next_u32()); }
    __device__ __forceinline__ double next_f64() { return philox::to_f64(next_u32()); }
    /* The next four draws as one vector (x first). */
    __device__ __forceinline__ uint4 next4()
    {
        uint4 r;
        r.x = next_u32(); r.y = next_u32(); r.z = next_u32(); r.w = next_u32();
        return r;
    }
    __device__ void store(const srng_dev_view &v, uint64_t stream) const
    {
        const uint64_t n = v.n_streams;
        v.tinymt_state[stream] = s0; v.tinymt_state[n + stream] = s1;
        v.tinymt_state[2 * n + stream] = s2; v.tinymt_state[3 * n + stream] = s3;
    }

    uint32_t s0, s1, s2, s3, mat1, mat2, tmat;
};

/* --------------------------------------------- non-uniform variates (FP32) */

/* Exponential and normal variates from the FP32 uniforms, computed with this
 * header's own elementary functions so that every machine that follows the
 * same IEEE-754 single operations (each product, sum, quotient and square root
 * rounded to nearest even; fused multiply-adds rounded once) gets the same
 * bits.  Every operation below is an explicit correctly rounded intrinsic, so
 * the compiler cannot contract or reorder it.  Accuracy: a few units in the
 * last place against the exact functions. */
namespace dist {

/* ln_unit: natural logarithm of x in (0, 1], Cody & Waite style.  x = 2^e m
 * with m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s), s = (m - 1) / (m + 1),
 * |s| <= 0.1716, by the odd series 2 (s + s^3/3 + ... + s^11/11) (truncation
 * below 2^-33 relative), its leading term 2s added last; ln x = e ln2 + ln m
 * with ln2 split into hi, its leading 15 bits (e hi is exact for |e| < 512),
 * and lo = ln2 - hi. */
__device__ __forceinline__ float ln_unit(float x)
{
    const uint32_t bits = __float_as_uint(x);
    int e = (int)((bits >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);  /* [1, 2) */
    if (m > 1.41421356237309504880f) { m = __fmul_rn(m, 0.5f); e += 1; }
    const float f = __fadd_rn(m, -1.0f);                              /* exact */
    const float sv = __fdiv_rn(f, __fadd_rn(m, 1.0f));
    const float z = __fmul_rn(sv, sv);
    float p = (float)(1.0 / 11.0);
    p = __fmaf_rn(p, z, (float)(1.0 / 9.0));
    p = __fmaf_rn(p, z, (float)(1.0 / 7.0));
    p = __fmaf_rn(p, z, (float)(1.0 / 5.0));
    p = __fmaf_rn(p, z, (float)(1.0 / 3.0));
    const float s2 = __fmul_rn(2.0f, sv);                              /* exact */
    const float lnm = __fmaf_rn(s2, __fmul_rn(z, p), s2);              /* leading term last */
    const float ef = (float)e;                                         /* |e| <= 150 */
    constexpr float kLn2Hi = 0.693145751953125f;                       /* 22713 / 2^15 */
    constexpr float kLn2Lo = (float)(0.69314718055994530942 - 0.693145751953125);
    return __fmaf_rn(ef, kLn2Hi, __fmaf_rn(ef, kLn2Lo, lnm));
}

/* Taylor coefficients of sin((pi/2) r) and cos((pi/2) r) in r:
 * coef(n) = (-1)^(n/2) (pi/2)^n / n!, evaluated in double, rounded once to float. */
namespace detail_sc {
constexpr double kHalfPi = 3.14159265358979323846 / 2.0;
constexpr double pw(int n) { return n == 0 ? 1.0 : kHalfPi * pw(n - 1); }
constexpr double fact(int n) { return n <= 1 ? 1.0 : n * fact(n - 1); }
constexpr float coef(int n) { return (float)(((n / 2) % 2 ? -1.0 : 1.0) * pw(n) / fact(n)); }
constexpr float kS1 = coef(1), kS3 = coef(3), kS5 = coef(5), kS7 = coef(7), kS9 = coef(9);
constexpr float kC2 = coef(2), kC4 = coef(4), kC6 = coef(6), kC8 = coef(8), kC10 = coef(10);
}  // namespace detail_sc

/* sin and cos of 2 pi u for u in [0, 1).  4u = q + r exactly (u has at most
 * 24 significant bits): q is the quadrant, r in [0, 1).  For r > 1/2 the
 * complement r' = 1 - r (exact) is used with sin and cos exchanged, so the
 * polynomials only see (pi/2) r' <= pi/4: sine to degree 9, cosine to degree
 * 10 (truncation below 2^-28), each with small relative error, also near the
 * zeros of sin and cos.  The quadrant then fixes signs and order. */
__device__ __forceinline__ void sincos_2pi(float u, float *s, float *c)
{
    using namespace detail_sc;
    const float v = __fmul_rn(u, 4.0f);
    const int q = (int)v;                                  /* 0..3 */
    float r = __fadd_rn(v, -(float)q);                     /* exact */
    const bool flip = r > 0.5f;
    if (flip) r = __fadd_rn(1.0f, -r);                     /* exact */
    const float r2 = __fmul_rn(r, r);
    float ps = kS9;
    ps = __fmaf_rn(ps, r2, kS7);
    ps = __fmaf_rn(ps, r2, kS5);
    ps = __fmaf_rn(ps, r2, kS3);
    ps = __fmaf_rn(ps, r2, kS1);
    float pc = kC10;
    pc = __fmaf_rn(pc, r2, kC8);
    pc = __fmaf_rn(pc, r2, kC6);
    pc = __fmaf_rn(pc, r2, kC4);
    pc = __fmaf_rn(pc, r2, kC2);
    const float sr = __fmul_rn(ps, r);
    const float cr = __fmaf_rn(pc, r2, 1.0f);
    const float sn = flip ? cr : sr, cs = flip ? sr : cr;  /* of (pi/2)(4u - q) */
    switch (q & 3) {
    case 0: *s = sn; *c = cs; break;
    case 1: *s = cs; *c = -sn; break;
    case 2: *s = -sn; *c = -cs; break;
    default: *s = -cs; *c = sn; break;
    }
}

/* Exponential(1) variate from an FP32 uniform u in [0, 1): -ln(1 - u).  For u
 * a multiple of 2^-24 (every FP32 output of the generators) 1 - u is exact. */
__device__ __forceinline__ float exponential(float u) { return __fsub_rn(0.0f, ln_unit(__fadd_rn(1.0f, -u))); }

/* Two standard normal variates from two FP32 uniforms (Box & Muller 1958):
 * r = sqrt(-2 ln(1 - u0)), t = 2 pi u1, (r cos t, r sin t). */
__device__ __forceinline__ void normal_pair(float u0, float u1, float *n0, float *n1)
{
    const float r = __fsqrt_rn(__fmul_rn(-2.0f, ln_unit(__fadd_rn(1.0f, -u0))));
    float s, c;
    sincos_2pi(u1, &s, &c);
    *n0 = __fmul_rn(r, c);
    *n1 = __fmul_rn(r, s);
}

}  // namespace dist

/* ----------------------------------------- the paper's Listing-1 form */

/* Compile-time interface check of a generator class (the paper's Sec. 6
 * checks, at compile time and without virtual calls, that every generator
 * provides its draw method and its state members): a device generator here
 * must provide next_u32 / next_f32 / next_f64 returning uint32_t / float /
 * double and store its state back with store(view, stream) or store(view). */
template <class G, class = void> struct is_generator : std::false_type {};
template <class G>
struct is_generator<G, std::void_t<decltype(std::declval<G &>().next_u32()), decltype(std::declval<G &>().next_f32()),
                                   decltype(std::declval<G &>().next_f64())>>
    : std::integral_constant<bool, std::is_same<decltype(std::declval<G &>().next_u32()), uint32_t>::value &&
                                       std::is_same<decltype(std::declval<G &>().next_f32()), float>::value &&
                                       std::is_same<decltype(std::declval<G &>().next_f64()), double>::value> {};
static_assert(is_generator<Mrg32k3a>::value, "Mrg32k3a must provide next_u32/next_f32/next_f64");
static_assert(is_generator<Philox4x32_10>::value, "Philox4x32_10 must provide next_u32/next_f32/next_f64");
static_assert(is_generator<Threefry4x32_20>::value, "Threefry4x32_20 must provide next_u32/next_f32/next_f64");
static_assert(is_generator<TinyMT32>::value, "TinyMT32 must provide next_u32/next_f32/next_f64");
static_assert(is_generator<Threefry4x64_20>::value, "Threefry4x64_20 must provide next_u32/next_f32/next_f64");
#if __cplusplus >= 202002L
template <class G>
concept DeviceGenerator = requires(G g) {
    { g.next_u32() } -> std::same_as<uint32_t>;
    { g.next_f32() } -> std::same_as<float>;
    { g.next_f64() } -> std::same_as<double>;
};
static_assert(DeviceGenerator<Mrg32k3a> && DeviceGenerator<Philox4x32_10> && DeviceGenerator<Threefry4x32_20> &&
              DeviceGenerator<Threefry4x64_20> && DeviceGenerator<TinyMT32>);
#endif

namespace detail {
/* The set bound by RNG<T, Gen>::init in this translation unit (internal
 * linkage: every .cu file that includes this header binds its own). */
static __constant__ srng_dev_view bound_view;

__device__ __forceinline__ uint64_t global_thread_index()
{
    const uint64_t block = (uint64_t)blockIdx.x + (uint64_t)gridDim.x * (blockIdx.y + (uint64_t)gridDim.y * blockIdx.z);
    const uint64_t tid = threadIdx.x + (uint64_t)blockDim.x * (threadIdx.y + (uint64_t)blockDim.y * threadIdx.z);
    return block * ((uint64_t)blockDim.x * blockDim.y * blockDim.z) + tid;
}

template <class T> struct draw;
template <> struct draw<uint32_t> { template <class G> __device__ static uint32_t f(G &g) { return g.next_u32(); } };
template <> struct draw<float> { template <class G> __device__ static float f(G &g) { return g.next_f32(); } };
template <> struct draw<double> { template <class G> __device__ static double f(G &g) { return g.next_f64(); } };

template <class Gen> struct gen_id;
template <> struct gen_id<Mrg32k3a> { static constexpr int value = SRNG_MRG32K3A; };
template <> struct gen_id<Philox4x32_10> { static constexpr int value = SRNG_PHILOX4X32_10; };
template <> struct gen_id<Threefry4x32_20> { static constexpr int value = SRNG_THREEFRY4X32_20; };
template <> struct gen_id<TinyMT32> { static constexpr int value = SRNG_TINYMT32; };
template <> struct gen_id<Threefry4x64_20> { static constexpr int value = SRNG_THREEFRY4X64_20; };
}  // namespace detail

/* The paper's device object (Listing 1): constructed inside a kernel with no
 * arguments, it picks up the stream of the calling thread -- stream number =
 * global thread index, blocks in grid order, threads in block order -- from
 * the set bound on the host by init(); next() returns the next value of type
 * T (uint32_t, float or double, with the fixed conversions of srng.h).  The
 * destructor stores the stream's state back, so the next kernel that uses
 * the set continues where this one stopped.  The bound set must have at
 * least as many streams as threads launched. */
template <class T, class Gen>
class RNG {
  public:
    __device__ RNG() : s_(detail::global_thread_index()), g_(detail::bound_view, s_) {}
    __device__ ~RNG()
    {
        if constexpr (detail::gen_id<Gen>::value == SRNG_MRG32K3A || detail::gen_id<Gen>::value == SRNG_TINYMT32)
            g_.store(detail::bound_view, s_);
        else g_.store(detail::bound_view);
    }
    __device__ __forceinline__ T next() { return detail::draw<T>::f(g_); }
    __device__ uint64_t stream() const { return s_; }

    /* Host set-up (Sec. 5.1): create a set of n_streams streams (one per thread
     * of the kernels to come) from `seed` and bind it.  The set is owned
     * until release(). */
    static srng_status init(uint64_t n_streams, uint64_t seed = 0x5EED5EED5EED5EEDull,
                            srng_spacing spacing = SRNG_SPACING_STREAM)
    {
        srng_set *s = nullptr;
        srng_status st = srng_create(&s, (srng_gen)detail::gen_id<Gen>::value, seed, n_streams, spacing, nullptr);
        if (st != SRNG_OK) return st;
        st = bind(s);
        if (st != SRNG_OK) { srng_destroy(s); return st; }
        owned() = s;
        return SRNG_OK;
    }
    /* Bind an existing set of the same generator (not owned). */
    static srng_status bind(const srng_set *set)
    {
        srng_dev_view v;
        srng_status st = srng_get_device_view(set, &v);
        if (st != SRNG_OK) return st;
        if (v.gen != detail::gen_id<Gen>::value) return SRNG_ERR_ARG;
        return cudaMemcpyToSymbol(detail::bound_view, &v, sizeof v) == cudaSuccess ? SRNG_OK : SRNG_ERR_CUDA;
    }
    /* Release (Sec. 5.1, Listing 1): destroy the set created by init(). */
    static srng_status release()
    {
        srng_status st = srng_destroy(owned());
        owned() = nullptr;
        return st;
    }
    static srng_set *set() { return owned(); }

  private:
    static srng_set *&owned()
    {
        static srng_set *s = nullptr;
        return s;
    }

  private:
    uint64_t s_;
    Gen g_;
};

}  // namespace srng

#endif /* SRNG_DEVICE_CUH */
