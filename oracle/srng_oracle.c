/*
 * srng_oracle.c -- plain, slow, obviously correct CPU oracle for the bulk
 * uniform-generation path of arXiv 1412.8266 (ShoveRand).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference leg load this file's library.  It shares
 * no code, header, table or constant generator with the CUDA library, and the
 * CUDA library never loads it.
 *
 * Every function is the plain definition of what it computes, written for a
 * reader who checks it against the paper by eye:
 *
 *   - MRG32k3a (paper Sec. 4.1, which cites L'Ecuyer 1999 for the generator):
 *     two order-3 multiple recursive components modulo m1 = 2^32-209 and
 *     m2 = 2^32-22853, a state of six integers, a period of about 2^191, and
 *     sequence splitting (Sec. 2.3) into 2^64 streams of 2^127 draws, each cut
 *     into substreams of 2^76 draws.  The recurrence coefficients are those of
 *     the cited publication; the paper itself does not print them.
 *   - Philox4x32-10 (paper Sec. 4.3, which cites Salmon et al. 2011): a
 *     counter-based generator whose parameter is a key; ten rounds of a
 *     multiply/xor network on a 4 x 32-bit counter with a 2 x 32-bit key.
 *   - The integer -> uniform conversions, the Monte Carlo quarter-circle hit
 *     test and the SplitMix64 seed expansion, which the paper leaves open; the
 *     readings taken are stated beside each function.
 *
 * Arithmetic: exact 64-bit (and, for the hit test, 128-bit) integers; the one
 * floating-point rounding (MRG32k3a -> double) is a single IEEE-754
 * round-to-nearest-even multiply, so the file is built with
 * -ffp-contract=off and without fast-math.
 *
 * Parallelism: the *_bulk and *_batch entry points split independent streams
 * or instances over OpenMP threads; each stream is still stepped one draw at a
 * time, in order.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------- */
/* MRG32k3a definition (Sec. 4.1; coefficients of L'Ecuyer 1999)           */
/* ---------------------------------------------------------------------- */

#define ORC_M1 4294967087ULL /* 2^32 - 209   */
#define ORC_M2 4294944443ULL /* 2^32 - 22853 */
#define ORC_A12 1403580LL    /* x1[n] =  a12 x1[n-2] - a13 x1[n-3]  mod m1 */
#define ORC_A13 810728LL
#define ORC_A21 527612LL     /* x2[n] =  a21 x2[n-1] - a23 x2[n-3]  mod m2 */
#define ORC_A23 1370589LL

enum { ORC_OUT_U32 = 0, ORC_OUT_F32 = 1, ORC_OUT_F64 = 2 };

/* State layout: s[0..2] = (x1[n-3], x1[n-2], x1[n-1]),
 *               s[3..5] = (x2[n-3], x2[n-2], x2[n-1]).
 * One step computes x1[n], x2[n], shifts them in, and returns the combined
 * value z = (x1[n] - x2[n]) mod m1, taken in [1, m1] (z = m1 when the two
 * components are equal).  Draw k of a stream is the value returned by step
 * k+1 from the stream's start state ("step, then output"). */
uint32_t oracle_mrg_step(uint32_t s[6])
{
    int64_t p1 = (ORC_A12 * (int64_t)s[1] - ORC_A13 * (int64_t)s[0]) % (int64_t)ORC_M1;
    if (p1 < 0) p1 += (int64_t)ORC_M1;
    s[0] = s[1]; s[1] = s[2]; s[2] = (uint32_t)p1;

    int64_t p2 = (ORC_A21 * (int64_t)s[5] - ORC_A23 * (int64_t)s[3]) % (int64_t)ORC_M2;
    if (p2 < 0) p2 += (int64_t)ORC_M2;
    s[3] = s[4]; s[4] = s[5]; s[5] = (uint32_t)p2;

    if (p1 > p2) return (uint32_t)(p1 - p2);
    return (uint32_t)(p1 - p2 + (int64_t)ORC_M1);
}

/* The one-step transition of each component as a 3x3 matrix acting on the
 * column (x[n-3], x[n-2], x[n-1]); entries reduced into [0, m). */
void oracle_mrg_matrix(int comp, uint64_t a[9])
{
    uint64_t m = comp == 0 ? ORC_M1 : ORC_M2;
    memset(a, 0, 9 * sizeof(uint64_t));
    a[0 * 3 + 1] = 1;
    a[1 * 3 + 2] = 1;
    if (comp == 0) {
        a[2 * 3 + 0] = m - (uint64_t)ORC_A13;
        a[2 * 3 + 1] = (uint64_t)ORC_A12;
    } else {
        a[2 * 3 + 0] = m - (uint64_t)ORC_A23;
        a[2 * 3 + 2] = (uint64_t)ORC_A21;
    }
}

/* c = a * b mod m for 3x3 matrices with entries in [0, m), m < 2^32. */
static void mat_mul(const uint64_t a[9], const uint64_t b[9], uint64_t m, uint64_t c[9])
{
    uint64_t t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            uint64_t acc = 0;
            for (int k = 0; k < 3; ++k)
                acc = (acc + (a[i * 3 + k] * b[k * 3 + j]) % m) % m;
            t[i * 3 + j] = acc;
        }
    memcpy(c, t, sizeof t);
}

/* out = A_comp^e mod m, e = e_hi * 2^64 + e_lo, by square-and-multiply. */
void oracle_mrg_matpow(int comp, uint64_t e_hi, uint64_t e_lo, uint64_t out[9])
{
    uint64_t m = comp == 0 ? ORC_M1 : ORC_M2;
    uint64_t base[9], r[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    oracle_mrg_matrix(comp, base);
    for (int bit = 0; bit < 128; ++bit) {
        uint64_t word = bit < 64 ? e_lo : e_hi;
        if ((word >> (bit & 63)) & 1) mat_mul(r, base, m, r);
        mat_mul(base, base, m, base);
    }
    memcpy(out, r, sizeof r);
}

/* v = a * v mod m for one component (3 entries). */
static void mat_vec(const uint64_t a[9], uint32_t v[3], uint64_t m)
{
    uint64_t t[3];
    for (int i = 0; i < 3; ++i) {
        uint64_t acc = 0;
        for (int k = 0; k < 3; ++k) acc = (acc + (a[i * 3 + k] * (uint64_t)v[k]) % m) % m;
        t[i] = acc;
    }
    for (int i = 0; i < 3; ++i) v[i] = (uint32_t)t[i];
}

/* Advance a state by n = n_hi * 2^64 + n_lo draws: s <- A^n s (Sec. 2.3,
 * sequence splitting; the jump is the n-th matrix power). */
void oracle_mrg_jump(uint32_t s[6], uint64_t n_hi, uint64_t n_lo)
{
    uint64_t a1[9], a2[9];
    oracle_mrg_matpow(0, n_hi, n_lo, a1);
    oracle_mrg_matpow(1, n_hi, n_lo, a2);
    mat_vec(a1, s, ORC_M1);
    mat_vec(a2, s + 3, ORC_M2);
}

/* Start states of `count` consecutive streams (Sec. 4.1: streams of 2^127
 * draws, substreams of 2^76).  Stream i starts 2^e draws after stream i-1;
 * stream 0 is the seed state.  Written out as the definition: step from the
 * seed state to stream `first`, then one jump of 2^e per following stream.
 * out holds 6 words per stream (same order as the state layout above). */
void oracle_mrg_stream_starts(const uint32_t seed_state[6], int e, uint64_t first, uint64_t count,
                              uint32_t *out)
{
    uint64_t j1[9], j2[9], f1[9], f2[9];
    uint64_t e_hi = e >= 64 ? (1ULL << (e - 64)) : 0;
    uint64_t e_lo = e >= 64 ? 0 : (1ULL << e);
    oracle_mrg_matpow(0, e_hi, e_lo, j1);           /* A1^(2^e) */
    oracle_mrg_matpow(1, e_hi, e_lo, j2);           /* A2^(2^e) */
    uint32_t y[6];
    memcpy(y, seed_state, sizeof y);
    /* stream `first` = (A^(2^e))^first applied to the seed state */
    uint64_t p1[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, p2[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    memcpy(f1, j1, sizeof f1);
    memcpy(f2, j2, sizeof f2);
    for (uint64_t k = first; k; k >>= 1) {
        if (k & 1) { mat_mul(p1, f1, ORC_M1, p1); mat_mul(p2, f2, ORC_M2, p2); }
        mat_mul(f1, f1, ORC_M1, f1);
        mat_mul(f2, f2, ORC_M2, f2);
    }
    mat_vec(p1, y, ORC_M1);
    mat_vec(p2, y + 3, ORC_M2);
    for (uint64_t i = 0; i < count; ++i) {
        memcpy(out + 6 * i, y, sizeof y);
        mat_vec(j1, y, ORC_M1);
        mat_vec(j2, y + 3, ORC_M2);
    }
}

/* A state is valid when every word of component c is below m_c and no
 * component is all zero (the all-zero component is a fixed point). */
int oracle_mrg_state_valid(const uint32_t s[6])
{
    for (int i = 0; i < 3; ++i) if (s[i] >= ORC_M1) return 0;
    for (int i = 3; i < 6; ++i) if (s[i] >= ORC_M2) return 0;
    if (s[0] == 0 && s[1] == 0 && s[2] == 0) return 0;
    if (s[3] == 0 && s[4] == 0 && s[5] == 0) return 0;
    return 1;
}

/* ---------------------------------------------------------------------- */
/* Seed expansion (the paper gives none; Sec. 2.3 only names seeding by     */
/* random statuses).  Reading: SplitMix64 (Steele, Lea & Flood, OOPSLA      */
/* 2014) seeded with the 64-bit seed; six successive outputs r0..r5 give    */
/* x1[i] = r_i mod m1 and x2[i] = r_(i+3) mod m2; a component that comes    */
/* out all zero is replaced by (12345, 12345, 12345).  Pinned against an     */
/* independent implementation of the same output mixer (tests).             */
/* ---------------------------------------------------------------------- */

uint64_t oracle_splitmix64_next(uint64_t *state)
{
    *state += 0x9E3779B97F4A7C15ULL;
    uint64_t z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void oracle_seed_expand(uint64_t seed, uint32_t out[6])
{
    uint64_t st = seed;
    uint64_t r[6];
    for (int i = 0; i < 6; ++i) r[i] = oracle_splitmix64_next(&st);
    for (int i = 0; i < 3; ++i) out[i] = (uint32_t)(r[i] % ORC_M1);
    for (int i = 0; i < 3; ++i) out[3 + i] = (uint32_t)(r[3 + i] % ORC_M2);
    if (out[0] == 0 && out[1] == 0 && out[2] == 0) out[0] = out[1] = out[2] = 12345;
    if (out[3] == 0 && out[4] == 0 && out[5] == 0) out[3] = out[4] = out[5] = 12345;
}

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 (Sec. 4.3; definition of Salmon et al. 2011)              */
/* ---------------------------------------------------------------------- */

#define ORC_PHILOX_M0 0xD2511F53U
#define ORC_PHILOX_M1 0xCD9E8D57U
#define ORC_PHILOX_W0 0x9E3779B9U /* floor(2^32 / golden ratio)   */
#define ORC_PHILOX_W1 0xBB67AE85U /* floor(2^32 * (sqrt(3) - 1))  */

/* One round: the two multiplies give (hi, lo) halves; the outputs are
 * (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0) with (hi0,lo0) = M0 * x0 and
 * (hi1,lo1) = M1 * x2.  Ten rounds, the key bumped by (W0, W1) between them. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += ORC_PHILOX_W0; k1 += ORC_PHILOX_W1; }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * x0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Word `p` of Philox stream `s` under key (k0, k1).  Reading of the paper's
 * "one key per thread" parameterisation as a counter split: the stream index
 * fills counter words 2-3, the block index q = p / 4 fills counter words
 * 0-1, and the draw is word p mod 4 of that block. */
uint32_t oracle_philox_word(uint32_t k0, uint32_t k1, uint64_t s, uint64_t p)
{
    uint64_t q = p / 4;
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), (uint32_t)s, (uint32_t)(s >> 32)};
    uint32_t key[2] = {k0, k1};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[p % 4];
}

/* ---------------------------------------------------------------------- */
/* Threefry4x32-20 (Sec. 4.3 names Threefry beside Philox, both from Salmon */
/* et al. 2011): the Threefish block structure on four 32-bit words.  Key   */
/* schedule: the four key words and a fifth, their xor with the parity     */
/* constant 0x1BD11BDA; subkey j adds key words (j, j+1, j+2, j+3) mod 5 to  */
/* the four state words and j to the last.  Subkey 0 is added first, then   */
/* after every fourth round the next subkey.  A round: MIX the word pairs   */
/* (0,1) and (2,3) -- a += b; b = (b <<< r) ^ a -- with the round's two     */
/* rotation counts (a cycle of eight pairs), then permute the words to      */
/* (0, 3, 2, 1).  Twenty rounds (the published default).                    */
/* PARITY UNPINNED: the rotation counts and the parity constant come from   */
/* the publication and no independent implementation is available here to */
/* compare with; only the structure is checked (see tests).                 */
/* ---------------------------------------------------------------------- */

static const int ORC_THREEFRY_ROT[8][2] = {
    {10, 26}, {11, 21}, {13, 27}, {23, 5}, {6, 20}, {17, 11}, {25, 10}, {18, 20}};
#define ORC_THREEFRY_PARITY 0x1BD11BDAU

static uint32_t orc_rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

void oracle_threefry4x32_20(const uint32_t ctr[4], const uint32_t key[4], uint32_t out[4])
{
    uint32_t ks[5];
    ks[4] = ORC_THREEFRY_PARITY;
    for (int i = 0; i < 4; ++i) {
        ks[i] = key[i];
        ks[4] ^= key[i];
    }
    uint32_t v[4];
    for (int i = 0; i < 4; ++i) v[i] = ctr[i] + ks[i];          /* subkey 0 */
    for (int d = 0; d < 20; ++d) {
        for (int pair = 0; pair < 2; ++pair) {                  /* MIX */
            uint32_t *a = &v[2 * pair], *b = &v[2 * pair + 1];
            *a = *a + *b;
            *b = orc_rotl32(*b, ORC_THREEFRY_ROT[d % 8][pair]) ^ *a;
        }
        uint32_t t = v[1];                                      /* permute (0, 3, 2, 1) */
        v[1] = v[3];
        v[3] = t;
        if (d % 4 == 3) {                                       /* subkey (d + 1) / 4 */
            uint32_t j = (uint32_t)(d + 1) / 4;
            for (int i = 0; i < 4; ++i) v[i] += ks[(j + i) % 5];
            v[3] += j;
        }
    }
    for (int i = 0; i < 4; ++i) out[i] = v[i];
}

/* Word p of Threefry stream s: the paper's per-thread key read literally --
 * key = (s low, s high, seed low, seed high), counter = (q low, q high, 0, 0)
 * with q = p / 4, the draw being word p mod 4 of that block. */
uint32_t oracle_threefry_word(uint64_t seed, uint64_t s, uint64_t p)
{
    uint64_t q = p / 4;
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), 0, 0};
    uint32_t key[4] = {(uint32_t)s, (uint32_t)(s >> 32), (uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_threefry4x32_20(ctr, key, out);
    return out[p % 4];
}

/* Threefry4x64-20: the same construction on four 64-bit words (the Threefish-
 * 256 block shape), parity constant 0x1BD11BDAA9FC1A22, the eight rotation
 * pairs below, twenty rounds.  PARITY UNPINNED for the constants, as for
 * Threefry4x32.  Stream layout: key = (s, seed, 0, 0), counter = (q, 0, 0, 0)
 * for block q; a block gives eight 32-bit draws, the low then the high half
 * of each word in order, so draw p is 32-bit word p mod 8 of block p / 8. */
static const int ORC_THREEFRY64_ROT[8][2] = {
    {14, 16}, {52, 57}, {23, 40}, {5, 37}, {25, 33}, {46, 12}, {58, 22}, {32, 32}};
#define ORC_THREEFRY64_PARITY 0x1BD11BDAA9FC1A22ULL

static uint64_t orc_rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

void oracle_threefry4x64_20(const uint64_t ctr[4], const uint64_t key[4], uint64_t out[4])
{
    uint64_t ks[5];
    ks[4] = ORC_THREEFRY64_PARITY;
    for (int i = 0; i < 4; ++i) {
        ks[i] = key[i];
        ks[4] ^= key[i];
    }
    uint64_t v[4];
    for (int i = 0; i < 4; ++i) v[i] = ctr[i] + ks[i];
    for (int d = 0; d < 20; ++d) {
        for (int pair = 0; pair < 2; ++pair) {
            uint64_t *a = &v[2 * pair], *b = &v[2 * pair + 1];
            *a = *a + *b;
            *b = orc_rotl64(*b, ORC_THREEFRY64_ROT[d % 8][pair]) ^ *a;
        }
        uint64_t t = v[1];
        v[1] = v[3];
        v[3] = t;
        if (d % 4 == 3) {
            uint64_t j = (uint64_t)(d + 1) / 4;
            for (int i = 0; i < 4; ++i) v[i] += ks[(j + i) % 5];
            v[3] += j;
        }
    }
    for (int i = 0; i < 4; ++i) out[i] = v[i];
}

uint32_t oracle_threefry64_word(uint64_t seed, uint64_t s, uint64_t p)
{
    uint64_t ctr[4] = {p / 8, 0, 0, 0};
    uint64_t key[4] = {s, seed, 0, 0};
    uint64_t out[4];
    oracle_threefry4x64_20(ctr, key, out);
    uint64_t w = out[(p % 8) / 2];
    return (p % 2) ? (uint32_t)(w >> 32) : (uint32_t)w;
}

/* ---------------------------------------------------------------------- */
/* Integer -> uniform conversions (fixed readings)                          */
/* ---------------------------------------------------------------------- */

/* 24-bit single: the top 24 bits of the word times 2^-24, in [0, 1). */
float oracle_to_f32(uint32_t v)
{
    return ldexpf((float)(v >> 8), -24);
}

/* MRG32k3a double: z * norm rounded once to nearest even, norm being the
 * double nearest 1/(m1+1); z in [1, m1] gives a value in (0, 1). */
double oracle_mrg_to_f64(uint32_t z)
{
    const double norm = 1.0 / 4294967088.0; /* 1 / (m1 + 1), one IEEE division */
    return (double)z * norm;
}

/* Philox double: (w + 1/2) * 2^-32, exact, in (0, 1). */
double oracle_philox_to_f64(uint32_t w)
{
    return ((double)w + 0.5) / 4294967296.0;
}

static void store_value(int out_type, void *out, uint64_t i, uint32_t v, int is_mrg)
{
    if (out_type == ORC_OUT_U32) ((uint32_t *)out)[i] = v;
    else if (out_type == ORC_OUT_F32) ((float *)out)[i] = oracle_to_f32(v);
    else ((double *)out)[i] = is_mrg ? oracle_mrg_to_f64(v) : oracle_philox_to_f64(v);
}

/* n draws of one MRG32k3a stream from state s (advanced in place). */
void oracle_mrg_generate(uint32_t s[6], uint64_t n, int out_type, void *out)
{
    for (uint64_t k = 0; k < n; ++k) store_value(out_type, out, k, oracle_mrg_step(s), 1);
}

/* n words of Philox stream s starting at position p. */
void oracle_philox_generate(uint32_t k0, uint32_t k1, uint64_t s, uint64_t p, uint64_t n,
                            int out_type, void *out)
{
    for (uint64_t k = 0; k < n; ++k) store_value(out_type, out, k, oracle_philox_word(k0, k1, s, p + k), 0);
}

/* n words of Threefry stream s starting at position p (conversions as Philox). */
void oracle_threefry_generate(uint64_t seed, uint64_t s, uint64_t p, uint64_t n, int out_type, void *out)
{
    for (uint64_t k = 0; k < n; ++k) store_value(out_type, out, k, oracle_threefry_word(seed, s, p + k), 0);
}

/* n draws of Threefry4x64 stream s starting at position p (conversions as Philox). */
void oracle_threefry64_generate(uint64_t seed, uint64_t s, uint64_t p, uint64_t n, int out_type, void *out)
{
    for (uint64_t k = 0; k < n; ++k) store_value(out_type, out, k, oracle_threefry64_word(seed, s, p + k), 0);
}

/* Stream-major bulk output of many streams:
 * out[i * n + k] = draw k of stream i.  MRG: states holds 6 words per stream
 * and is advanced in place.  Philox: positions[i] is the start position of
 * stream (stream0 + i) and is advanced by n. */
void oracle_mrg_bulk(uint32_t *states, uint64_t n_streams, uint64_t n, int out_type, void *out,
                     int threads)
{
    size_t esz = out_type == ORC_OUT_F64 ? 8 : 4;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < (int64_t)n_streams; ++i)
        oracle_mrg_generate(states + 6 * i, n, out_type, (char *)out + (size_t)i * n * esz);
}

void oracle_philox_bulk(uint32_t k0, uint32_t k1, uint64_t stream0, uint64_t *positions,
                        uint64_t n_streams, uint64_t n, int out_type, void *out, int threads)
{
    size_t esz = out_type == ORC_OUT_F64 ? 8 : 4;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < (int64_t)n_streams; ++i) {
        oracle_philox_generate(k0, k1, stream0 + (uint64_t)i, positions[i], n, out_type,
                               (char *)out + (size_t)i * n * esz);
        positions[i] += n;
    }
}

void oracle_threefry_bulk(uint64_t seed, uint64_t stream0, uint64_t *positions, uint64_t n_streams,
                          uint64_t n, int out_type, void *out, int threads)
{
    size_t esz = out_type == ORC_OUT_F64 ? 8 : 4;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < (int64_t)n_streams; ++i) {
        oracle_threefry_generate(seed, stream0 + (uint64_t)i, positions[i], n, out_type,
                                 (char *)out + (size_t)i * n * esz);
        positions[i] += n;
    }
}

void oracle_threefry64_bulk(uint64_t seed, uint64_t stream0, uint64_t *positions, uint64_t n_streams,
                            uint64_t n, int out_type, void *out, int threads)
{
    size_t esz = out_type == ORC_OUT_F64 ? 8 : 4;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < (int64_t)n_streams; ++i) {
        oracle_threefry64_generate(seed, stream0 + (uint64_t)i, positions[i], n, out_type,
                                   (char *)out + (size_t)i * n * esz);
        positions[i] += n;
    }
}

/* ---------------------------------------------------------------------- */
/* Monte Carlo quarter-circle hit count (fused consumer reading).          */
/* Draws are taken in pairs (2k, 2k+1), k < floor(L/2); a pair hits when    */
/* the point lies strictly inside the quarter disc, tested exactly on the   */
/* defined uniforms:                                                        */
/*   Philox: u = (w >> 8) 2^-24   ->  a^2 + b^2 < 2^48                      */
/*   MRG   : u = z / (m1 + 1)     ->  z1^2 + z2^2 < (m1 + 1)^2              */
/* ---------------------------------------------------------------------- */

int oracle_pi_hit_philox(uint32_t w0, uint32_t w1)
{
    unsigned __int128 a = w0 >> 8, b = w1 >> 8;
    return a * a + b * b < ((unsigned __int128)1 << 48);
}

int oracle_pi_hit_mrg(uint32_t z0, uint32_t z1)
{
    unsigned __int128 a = z0, b = z1, r = ORC_M1 + 1;
    return a * a + b * b < r * r;
}

int64_t oracle_mrg_pi_count(uint32_t s[6], uint64_t length)
{
    int64_t hits = 0;
    for (uint64_t k = 0; k + 1 < length; k += 2) {
        uint32_t z0 = oracle_mrg_step(s);
        uint32_t z1 = oracle_mrg_step(s);
        hits += oracle_pi_hit_mrg(z0, z1);
    }
    if (length & 1) (void)oracle_mrg_step(s); /* the unpaired last draw is consumed, not used */
    return hits;
}

int64_t oracle_philox_pi_count(uint32_t k0, uint32_t k1, uint64_t s, uint64_t p, uint64_t length)
{
    int64_t hits = 0;
    for (uint64_t k = 0; k + 1 < length; k += 2)
        hits += oracle_pi_hit_philox(oracle_philox_word(k0, k1, s, p + k),
                                     oracle_philox_word(k0, k1, s, p + k + 1));
    return hits;
}

int64_t oracle_threefry64_pi_count(uint64_t seed, uint64_t s, uint64_t p, uint64_t length)
{
    int64_t hits = 0;
    for (uint64_t k = 0; k + 1 < length; k += 2)
        hits += oracle_pi_hit_philox(oracle_threefry64_word(seed, s, p + k), oracle_threefry64_word(seed, s, p + k + 1));
    return hits;
}

/* Threefry words take the Philox hit test (the same 24-bit single reading). */
int64_t oracle_threefry_pi_count(uint64_t seed, uint64_t s, uint64_t p, uint64_t length)
{
    int64_t hits = 0;
    for (uint64_t k = 0; k + 1 < length; k += 2)
        hits += oracle_pi_hit_philox(oracle_threefry_word(seed, s, p + k), oracle_threefry_word(seed, s, p + k + 1));
    return hits;
}

/* ---------------------------------------------------------------------- */
/* Batched instances: instance i draws `lengths[i]` values from its own     */
/* stream.  gens[i] = 0 for MRG32k3a (start state in mrg_states, 6 words    */
/* per instance, not modified), 1 for Philox (stream philox_streams[i] from */
/* position philox_pos[i] under key (k0, k1)), 3 for Threefry (the same     */
/* stream and position, seed k0 + 2^32 k1).                                 */
/* mode 0: u32 output written at out_offsets[i]; mode 1: hit counts.        */
/* ---------------------------------------------------------------------- */

void oracle_batch(uint64_t n_inst, const int32_t *gens, const uint32_t *mrg_states,
                  uint32_t k0, uint32_t k1, const uint64_t *philox_streams,
                  const uint64_t *philox_pos, const uint64_t *lengths,
                  const uint64_t *out_offsets, int mode, int out_type, void *out,
                  int64_t *counts, int threads)
{
    size_t esz = out_type == ORC_OUT_F64 ? 8 : 4;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < (int64_t)n_inst; ++i) {
        if (gens[i] == 0) {
            uint32_t s[6];
            memcpy(s, mrg_states + 6 * i, sizeof s);
            if (mode == 0)
                oracle_mrg_generate(s, lengths[i], out_type, (char *)out + out_offsets[i] * esz);
            else
                counts[i] = oracle_mrg_pi_count(s, lengths[i]);
        } else if (gens[i] == 3) {
            uint64_t seed = (uint64_t)k1 << 32 | k0;
            if (mode == 0)
                oracle_threefry_generate(seed, philox_streams[i], philox_pos[i], lengths[i], out_type,
                                         (char *)out + out_offsets[i] * esz);
            else
                counts[i] = oracle_threefry_pi_count(seed, philox_streams[i], philox_pos[i], lengths[i]);
        } else {
            if (mode == 0)
                oracle_philox_generate(k0, k1, philox_streams[i], philox_pos[i], lengths[i],
                                       out_type, (char *)out + out_offsets[i] * esz);
            else
                counts[i] = oracle_philox_pi_count(k0, k1, philox_streams[i], philox_pos[i],
                                                   lengths[i]);
        }
    }
}

/* ---------------------------------------------------------------------- */
/* TinyMT32 (Sec. 4.2; Saito & Matsumoto 2011): a 127-bit GF(2)-linear      */
/* state of four 32-bit words (bit 31 of word 0 unused), parameterised by   */
/* (mat1, mat2, tmat).  One step:                                           */
/*   x = (s0 & 0x7fffffff) ^ s1 ^ s2;  x ^= x << 1;                         */
/*   y = s3 ^ (s3 >> 1) ^ x;                                                 */
/*   (s0, s1, s2, s3) = (s1, s2, x ^ (y << 10), y), then if y is odd         */
/*   s1 ^= mat1 and s2 ^= mat2.                                             */
/* Output (tempering): t = s0 + (s2 >> 8); v = s3 ^ t, ^ tmat if t is odd.   */
/* Seeding of a parameter set from a 32-bit seed: (seed, mat1, mat2, tmat),  */
/* words 1..7 (mod 4) mixed with i + 1812433253 (w ^ (w >> 30)) of the       */
/* previous word, an all-zero state replaced by 'T','I','N','Y', then eight  */
/* steps.  The paper's hybrid (Sec. 4.2): one parameter set per group of     */
/* streams (a CUDA block), and stream j of a group starts j * 2^64 steps    */
/* after the group's seed state (sequence splitting).                        */
/* Jumps use the characteristic polynomial p of the step (degree 127, found */
/* by Berlekamp-Massey on an output bit of the state): T^J s = r(T) s with  */
/* r = x^J mod p, evaluated by Horner's rule on states.                     */
/* Parity: the step is pinned (maximal period of the authors' default set,  */
/* checked with sympy), the seeding's mixing function against numpy's      */
/* MT19937 initialisation; the tempering is PARITY UNPINNED (structure only).*/
/* ---------------------------------------------------------------------- */

#define ORC_TMT_MASK 0x7fffffffU

void oracle_tinymt32_next(uint32_t s[4], uint32_t mat1, uint32_t mat2)
{
    uint32_t x = (s[0] & ORC_TMT_MASK) ^ s[1] ^ s[2];
    x ^= x << 1;
    uint32_t y = s[3] ^ (s[3] >> 1) ^ x;
    s[0] = s[1];
    s[1] = s[2];
    s[2] = x ^ (y << 10);
    s[3] = y;
    if (y & 1) {
        s[1] ^= mat1;
        s[2] ^= mat2;
    }
}

uint32_t oracle_tinymt32_temper(const uint32_t s[4], uint32_t tmat)
{
    uint32_t t = s[0] + (s[2] >> 8);
    uint32_t v = s[3] ^ t;
    if (t & 1) v ^= tmat;
    return v;
}

void oracle_tinymt32_init(uint32_t seed32, uint32_t mat1, uint32_t mat2, uint32_t tmat, uint32_t s[4])
{
    s[0] = seed32;
    s[1] = mat1;
    s[2] = mat2;
    s[3] = tmat;
    for (uint32_t i = 1; i < 8; ++i) {
        uint32_t prev = s[(i - 1) % 4];
        s[i % 4] ^= i + 1812433253U * (prev ^ (prev >> 30));
    }
    if ((s[0] & ORC_TMT_MASK) == 0 && s[1] == 0 && s[2] == 0 && s[3] == 0) {
        s[0] = 'T';
        s[1] = 'I';
        s[2] = 'N';
        s[3] = 'Y';
    }
    for (int i = 0; i < 8; ++i) oracle_tinymt32_next(s, mat1, mat2);
}

/* Polynomials over GF(2) as coefficient arrays: c[i] = coefficient of x^i. */
#define ORC_PMAX 256

/* Characteristic polynomial of the step: minimal polynomial (Berlekamp-
 * Massey) of bit 0 of s3 along 2 x 127 steps from the parameter set's seed-1
 * state.  Returns its degree L; p[0..L] receives the coefficients. */
int oracle_tinymt32_charpoly(uint32_t mat1, uint32_t mat2, uint8_t p[ORC_PMAX])
{
    uint8_t bits[254];
    uint32_t s[4];
    oracle_tinymt32_init(1, mat1, mat2, 0, s);
    for (int i = 0; i < 254; ++i) {
        oracle_tinymt32_next(s, mat1, mat2);
        bits[i] = s[3] & 1;
    }
    uint8_t c[ORC_PMAX] = {0}, b[ORC_PMAX] = {0}, t[ORC_PMAX];
    c[0] = b[0] = 1;
    int L = 0, m = 1;
    for (int n = 0; n < 254; ++n) {
        int d = bits[n];
        for (int i = 1; i <= L; ++i) d ^= c[i] & bits[n - i];
        if (!d) {
            ++m;
        } else if (2 * L <= n) {
            memcpy(t, c, sizeof t);
            for (int i = 0; i + m < ORC_PMAX; ++i) c[i + m] ^= b[i];
            L = n + 1 - L;
            memcpy(b, t, sizeof b);
            m = 1;
        } else {
            for (int i = 0; i + m < ORC_PMAX; ++i) c[i + m] ^= b[i];
            ++m;
        }
    }
    memset(p, 0, ORC_PMAX);
    for (int i = 0; i <= L; ++i) p[L - i] = c[i];   /* reciprocal of the connection polynomial */
    return L;
}

/* a * b mod p, all of degree < 127 except p (degree 127). */
static void orc_pmulmod(const uint8_t a[128], const uint8_t b[128], const uint8_t p[ORC_PMAX], uint8_t out[128])
{
    uint8_t prod[256] = {0};
    for (int i = 0; i < 127; ++i)
        if (a[i])
            for (int j = 0; j < 127; ++j) prod[i + j] ^= b[j];
    for (int k = 252; k >= 127; --k)
        if (prod[k])
            for (int i = 0; i <= 127; ++i) prod[k - 127 + i] ^= p[i];
    memcpy(out, prod, 128);
}

/* r = x^J mod p for J = (e_hi, e_lo), by left-to-right square and multiply. */
static void orc_xpow(uint64_t e_hi, uint64_t e_lo, const uint8_t p[ORC_PMAX], uint8_t r[128])
{
    memset(r, 0, 128);
    r[0] = 1;
    uint8_t x[128] = {0};
    x[1] = 1;
    for (int bit = 127; bit >= 0; --bit) {
        orc_pmulmod(r, r, p, r);
        uint64_t word = bit >= 64 ? e_hi : e_lo;
        if ((word >> (bit % 64)) & 1) orc_pmulmod(r, x, p, r);
    }
}

/* 1 when the step has period 2^127 - 1: p of degree 127 divides x^(2^127) - x
 * and has no root in GF(2); 127 being prime, p is then irreducible, and
 * 2^127 - 1 being prime, primitive. */
int oracle_tinymt32_max_period(uint32_t mat1, uint32_t mat2)
{
    uint8_t p[ORC_PMAX];
    if (oracle_tinymt32_charpoly(mat1, mat2, p) != 127) return 0;
    int ones = 0;
    for (int i = 0; i <= 127; ++i) ones += p[i];
    if (p[0] == 0 || ones % 2 == 0) return 0;   /* x or x + 1 divides p */
    uint8_t r[128] = {0};
    r[1] = 1;
    for (int i = 0; i < 127; ++i) orc_pmulmod(r, r, p, r);   /* x^(2^127) */
    for (int i = 0; i < 128; ++i)
        if (r[i] != (i == 1)) return 0;
    return 1;
}

/* Parameter sets with period 2^127 - 1 drawn from SplitMix64(seed): each
 * candidate takes two outputs a, b: mat1 = a mod 2^32, mat2 = a >> 32,
 * tmat = b mod 2^32 (the tempering parameter is not tuned for
 * equidistribution; it does not enter the period).  out[3 i + 0..2]. */
void oracle_tinymt32_find_params(uint64_t seed, uint32_t count, uint32_t *out)
{
    uint64_t sm = seed;
    uint32_t found = 0;
    while (found < count) {
        uint64_t a = oracle_splitmix64_next(&sm);
        uint64_t b = oracle_splitmix64_next(&sm);
        uint32_t mat1 = (uint32_t)a, mat2 = (uint32_t)(a >> 32), tmat = (uint32_t)b;
        if (!oracle_tinymt32_max_period(mat1, mat2)) continue;
        out[3 * found] = mat1;
        out[3 * found + 1] = mat2;
        out[3 * found + 2] = tmat;
        ++found;
    }
}

/* s <- T^J s for J = (e_hi, e_lo) (s must come from at least one step). */
void oracle_tinymt32_jump(uint32_t s[4], uint32_t mat1, uint32_t mat2, uint64_t e_hi, uint64_t e_lo)
{
    uint8_t p[ORC_PMAX], r[128];
    oracle_tinymt32_charpoly(mat1, mat2, p);
    orc_xpow(e_hi, e_lo, p, r);
    uint32_t acc[4] = {0, 0, 0, 0};
    for (int i = 126; i >= 0; --i) {
        oracle_tinymt32_next(acc, mat1, mat2);
        if (r[i])
            for (int w = 0; w < 4; ++w) acc[w] ^= s[w];
    }
    memcpy(s, acc, sizeof acc);
}

/* Start state of stream j of a group: the group's seed state (seed32 and its
 * parameters), then j * 2^64 steps. */
void oracle_tinymt32_stream_start(uint32_t seed32, const uint32_t prm[3], uint64_t j, uint32_t s[4])
{
    oracle_tinymt32_init(seed32, prm[0], prm[1], prm[2], s);
    if (j) oracle_tinymt32_jump(s, prm[0], prm[1], j, 0);   /* J = j * 2^64 */
}

/* Start states of n_streams streams, stream i in group i / group_size:
 * the group's seed state, then each next stream of the group 2^64 steps
 * after the previous one (r = x^(2^64) mod p applied once per stream).
 * out[4 i .. 4 i + 3]; prm[3 g .. 3 g + 2] per group. */
void oracle_tinymt32_stream_starts(uint32_t seed32, const uint32_t *prm, uint64_t group_size, uint64_t n_streams,
                                   uint32_t *out)
{
    uint64_t n_groups = (n_streams + group_size - 1) / group_size;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t g = 0; g < (int64_t)n_groups; ++g) {
        const uint32_t *p = prm + 3 * g;
        uint8_t poly[ORC_PMAX], r[128];
        oracle_tinymt32_charpoly(p[0], p[1], poly);
        orc_xpow(1, 0, poly, r);                       /* x^(2^64) mod p */
        uint32_t s[4];
        oracle_tinymt32_init(seed32, p[0], p[1], p[2], s);
        for (uint64_t j = 0; j < group_size && g * group_size + j < n_streams; ++j) {
            if (j > 0) {                               /* s <- r(T) s */
                uint32_t acc[4] = {0, 0, 0, 0};
                for (int i = 126; i >= 0; --i) {
                    oracle_tinymt32_next(acc, p[0], p[1]);
                    if (r[i])
                        for (int w = 0; w < 4; ++w) acc[w] ^= s[w];
                }
                memcpy(s, acc, sizeof acc);
            }
            memcpy(out + 4 * (g * group_size + j), s, sizeof s);
        }
    }
}

/* n draws of one stream from state s (advanced in place): step, then temper. */
void oracle_tinymt32_generate(uint32_t s[4], const uint32_t prm[3], uint64_t n, int out_type, void *out)
{
    for (uint64_t k = 0; k < n; ++k) {
        oracle_tinymt32_next(s, prm[0], prm[1]);
        store_value(out_type, out, k, oracle_tinymt32_temper(s, prm[2]), 0);
    }
}

/* Stream-major bulk output; stream i uses parameter set i / group_size and
 * its state states[4 i .. 4 i + 3] (advanced in place). */
void oracle_tinymt32_bulk(uint32_t *states, const uint32_t *prm, uint64_t group_size, uint64_t n_streams,
                          uint64_t n, int out_type, void *out, int threads)
{
    size_t esz = out_type == ORC_OUT_F64 ? 8 : 4;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < (int64_t)n_streams; ++i)
        oracle_tinymt32_generate(states + 4 * i, prm + 3 * ((uint64_t)i / group_size), n, out_type,
                                 (char *)out + (size_t)i * n * esz);
}

/* ---------------------------------------------------------------------- */
/* Non-uniform variates from FP32 uniforms (beyond the paper, which covers  */
/* uniform draws only): exponential by inversion, normal by Box & Muller    */
/* (1958).  The reading taken: single precision throughout, every step one  */
/* correctly rounded IEEE single operation or fused multiply-add, so that a */
/* device following the same steps agrees bit for bit.  ln, sin and cos are */
/* written out here from their series, not taken from libm:                 */
/*   ln x  = e ln2 + 2 atanh(s), x = 2^e m, m in [sqrt(1/2), sqrt(2)],      */
/*           s = (m-1)/(m+1), atanh(s) = s + s^3/3 + ... + s^11/11, the     */
/*           leading 2s added last,                                         */
/*           ln2 = hi + lo, hi = its leading 15 bits (Cody & Waite 1980);   */
/*   sin/cos(2 pi u): 4u = q + r, quadrant q, r in [0,1), r -> 1 - r with   */
/*           sin and cos exchanged when r > 1/2, then the Taylor series of  */
/*           sin((pi/2) r) to r^9 and cos((pi/2) r) to r^10.               */
/* Domain: uniforms in [0, 1).                                              */
/* ---------------------------------------------------------------------- */

typedef struct {
    float ln2_hi, ln2_lo;
    float inv_odd[6];   /* 1/1, 1/3, ..., 1/11 */
    float sc[11];       /* sc[n] = (-1)^floor(n/2) (pi/2)^n / n!, n = 1..10 */
} orc_dist_k;

static void orc_dist_init(orc_dist_k *k)
{
    const double ln2 = log(2.0);
    const double hi = ldexp(floor(ldexp(ln2, 15)), -15);
    k->ln2_hi = (float)hi;
    k->ln2_lo = (float)(ln2 - hi);
    for (int j = 0; j < 6; ++j) k->inv_odd[j] = 1.0f / (float)(2 * j + 1);
    /* (pi/2)^n / n! by the ratio of successive terms: t_n = t_(n-1) (pi/2) / n */
    const double half_pi = acos(-1.0) / 2.0;
    double t = 1.0;
    k->sc[0] = 1.0f;
    for (int n = 1; n <= 10; ++n) {
        t = t * half_pi / (double)n;
        k->sc[n] = (float)(((n / 2) % 2) ? -t : t);
    }
}

/* The constants as used: out[0] = ln2 hi, out[1] = ln2 lo,
 * out[2 + j] = 1/(2j+1) for j = 0..5, out[8 + n - 1] = sc[n] for n = 1..10. */
void oracle_dist_constants(float out[18])
{
    orc_dist_k k;
    orc_dist_init(&k);
    out[0] = k.ln2_hi;
    out[1] = k.ln2_lo;
    for (int j = 0; j < 6; ++j) out[2 + j] = k.inv_odd[j];
    for (int n = 1; n <= 10; ++n) out[8 + n - 1] = k.sc[n];
}

static float orc_ln(const orc_dist_k *k, float x)
{
    uint32_t bits;
    memcpy(&bits, &x, 4);
    int e = (int)((bits >> 23) & 0xFFu) - 127;
    uint32_t mbits = (bits & 0x007FFFFFu) | 0x3F800000u;   /* m in [1, 2) */
    float m;
    memcpy(&m, &mbits, 4);
    if ((double)m * (double)m > 2.0) {                      /* m > sqrt 2 */
        m = m * 0.5f;
        e = e + 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float p = k->inv_odd[5];
    for (int j = 4; j >= 1; --j) p = fmaf(p, s2, k->inv_odd[j]);
    /* 2 atanh(s) = 2s + 2s (s^2/3 + s^4/5 + ... + s^10/11) */
    float ln_m = fmaf(2.0f * s, s2 * p, 2.0f * s);
    float ef = (float)e;
    return fmaf(ef, k->ln2_hi, fmaf(ef, k->ln2_lo, ln_m));
}

static void orc_sincos_2pi(const orc_dist_k *k, float u, float *sin_out, float *cos_out)
{
    float v = u * 4.0f;
    int q = (int)v;
    float r = v - (float)q;
    int exchanged = r > 0.5f;
    if (exchanged) r = 1.0f - r;
    float r2 = r * r;
    float ps = k->sc[9];
    for (int n = 7; n >= 1; n -= 2) ps = fmaf(ps, r2, k->sc[n]);
    float pc = k->sc[10];
    for (int n = 8; n >= 2; n -= 2) pc = fmaf(pc, r2, k->sc[n]);
    float sin_r = ps * r;                 /* sin((pi/2) r) */
    float cos_r = fmaf(pc, r2, 1.0f);     /* cos((pi/2) r) */
    float sn = exchanged ? cos_r : sin_r;
    float cs = exchanged ? sin_r : cos_r;
    /* sin and cos of q pi/2 + phi */
    if (q % 4 == 0) { *sin_out = sn; *cos_out = cs; }
    else if (q % 4 == 1) { *sin_out = cs; *cos_out = -sn; }
    else if (q % 4 == 2) { *sin_out = -sn; *cos_out = -cs; }
    else { *sin_out = -cs; *cos_out = sn; }
}

float oracle_ln_unit_f32(float x)
{
    orc_dist_k k;
    orc_dist_init(&k);
    return orc_ln(&k, x);
}

void oracle_sincos_2pi_f32(float u, float *s, float *c)
{
    orc_dist_k k;
    orc_dist_init(&k);
    orc_sincos_2pi(&k, u, s, c);
}

void oracle_sincos_2pi_array(const float *u, uint64_t n, float *s, float *c)
{
    orc_dist_k k;
    orc_dist_init(&k);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) orc_sincos_2pi(&k, u[i], &s[i], &c[i]);
}

enum { ORC_DIST_EXPONENTIAL = 0, ORC_DIST_NORMAL = 1 };

/* dist 0: out[i] = -ln(1 - in[i]);
 * dist 1: out[2j] = r cos t, out[2j+1] = r sin t with
 *         r = sqrt(-2 ln(1 - in[2j])), t = 2 pi in[2j+1]   (n even). */
void oracle_transform(int dist, const float *in, uint64_t n, float *out)
{
    orc_dist_k k;
    orc_dist_init(&k);
    if (dist == ORC_DIST_EXPONENTIAL) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = 0.0f - orc_ln(&k, 1.0f - in[i]);
    } else {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < (int64_t)(n / 2); ++j) {
            float r = sqrtf(-2.0f * orc_ln(&k, 1.0f - in[2 * j]));
            float s, c;
            orc_sincos_2pi(&k, in[2 * j + 1], &s, &c);
            out[2 * j] = r * c;
            out[2 * j + 1] = r * s;
        }
    }
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
