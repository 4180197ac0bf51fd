/*
 * srng.h -- C ABI of the GB300 bulk uniform-generation library.
 *
 * The library implements the hot path of arXiv 1412.8266 (Passerat-Palmbach &
 * Hill, "How to correctly deal with pseudorandom numbers in manycore
 * environments", ShoveRand): many independent, reproducible streams of
 * uniform pseudorandom numbers on the GPU, one stream per processing element.
 *
 *   - MRG32k3a (paper Sec. 4.1): 2^64 streams of 2^127 draws, each cut into
 *     substreams of 2^76 draws, placed by sequence splitting (Sec. 2.3) with
 *     3x3 jump-ahead matrix powers modulo m1 = 2^32-209 and m2 = 2^32-22853.
 *   - Philox4x32-10 (paper Sec. 4.3): counter-based; the parameter is a key.
 *   - Threefry4x32-20 and Threefry4x64-20 (named beside Philox in Sec. 4.3):
 *     counter-based, add / rotate / xor rounds, key = (stream, seed).
 *   - TinyMT32 (Sec. 4.2): a parameter set shared by a group of streams,
 *     substreams 2^64 apart by polynomial jump-ahead.
 *   - Exponential and normal variates from the FP32 uniforms (srng_transform,
 *     and fused into generation as SRNG_OUT_EXP_F32 / SRNG_OUT_NORMAL_F32).
 *
 * Host set-up (paper Sec. 5.1: one host call allocates and places the streams
 * before the kernels run) maps to srng_create; release (Sec. 5, Listing 1)
 * maps to srng_destroy; the device-side constructor + next() (Sec. 5.2) is the
 * device header srng_device.cuh.
 *
 * Conventions shared by every entry point:
 *   - Pointers named *_dev are device pointers (cudaMalloc, torch, or any
 *     allocation the current device can address).  Pointers named *_host are
 *     host pointers (pinned memory gives the fastest copies).
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it unless the entry point
 *     says it synchronises.
 *   - Every call returns an srng_status; on failure srng_last_error() returns a
 *     message (per host thread) and nothing was enqueued unless stated.
 *   - Output layout of every generate call is stream-major and contiguous:
 *     out[(s - stream_begin) * n_per_stream + k] = draw k of stream s, counted
 *     from the stream's position when the call is made.  Values never depend
 *     on launch configuration or tuning.
 *   - Output of the uniform types (fixed conversions):
 *       SRNG_OUT_U32: MRG32k3a z = (x1 - x2) mod m1 taken in [1, m1]
 *                     (0 and values above m1 never occur); Philox, Threefry,
 *                     TinyMT32: the 32-bit word.
 *       SRNG_OUT_F32: (v >> 8) * 2^-24, exact, in [0, 1) (every generator).
 *       SRNG_OUT_F64: MRG32k3a: z * norm rounded to nearest even, norm the
 *                     double nearest 1/(m1+1), in (0, 1);
 *                     the others: (2w + 1) * 2^-33, exact, in (0, 1).
 */
#ifndef SRNG_H
#define SRNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SRNG_ABI_VERSION 3

typedef enum srng_status {
    SRNG_OK = 0,
    SRNG_ERR_ARG = 1,      /* invalid argument: NULL pointer, zero/too large count, bad enum   */
    SRNG_ERR_OOM = 2,      /* a device or host allocation failed                              */
    SRNG_ERR_STATE = 3,    /* an explicit MRG32k3a state violates 0 <= x < m / non-zero rule   */
    SRNG_ERR_CUDA = 4,     /* a CUDA runtime call failed; srng_last_error() has its message    */
    SRNG_ERR_BUDGET = 5,   /* a request is larger than the server's whole memory budget        */
    SRNG_ERR_TIMEOUT = 6,  /* a bounded wait expired                                           */
    SRNG_ERR_RANGE = 7,    /* stream range outside the set, or a position would overflow       */
    SRNG_ERR_CLOSED = 8,   /* the server is stopped / the ticket is unknown                    */
    SRNG_ERR_UNSUPPORTED = 9 /* operation not defined for this generator                       */
} srng_status;

typedef enum srng_gen {
    SRNG_MRG32K3A = 0,
    SRNG_PHILOX4X32_10 = 1,      /* streams split the counter, one key per set        */
    SRNG_PHILOX4X32_10_KEYED = 2, /* one key per stream (paper Sec. 4.3): see srng_create */
    SRNG_THREEFRY4X32_20 = 3,     /* Threefry4x32, 20 rounds (Sec. 4.3): see srng_create  */
    SRNG_TINYMT32 = 4,            /* TinyMT32 (Sec. 4.2): see srng_create_tinymt          */
    SRNG_THREEFRY4X64_20 = 5      /* Threefry4x64, 20 rounds (Sec. 4.3): see srng_create  */
} srng_gen;

typedef enum srng_out {
    SRNG_OUT_U32 = 0,
    SRNG_OUT_F32 = 1,
    SRNG_OUT_F64 = 2,
    /* Fused non-uniform variates (bulk generation calls only; see srng_transform
     * for the functions, which these outputs apply in the generation kernel):
     *   SRNG_OUT_EXP_F32: exponential(FP32 uniform of draw k);
     *   SRNG_OUT_NORMAL_F32: Box-Muller on pairs of draws.  Philox / Threefry:
     *     the pairs are the stream positions (2j, 2j + 1) -- value at position
     *     P is component P mod 2 (0: r cos t, 1: r sin t) of pair P / 2, any
     *     start and length.  MRG32k3a / TinyMT32: the pairs are draws
     *     (2i, 2i + 1) of the call; n must be even.                          */
    SRNG_OUT_EXP_F32 = 3,
    SRNG_OUT_NORMAL_F32 = 4
} srng_out;

/* Spacing of consecutive streams of an MRG32k3a set (paper Sec. 4.1). */
typedef enum srng_spacing {
    SRNG_SPACING_STREAM = 0,    /* 2^127 draws apart */
    SRNG_SPACING_SUBSTREAM = 1  /* 2^76 draws apart  */
} srng_spacing;

/* Unit of a jump distance. */
typedef enum srng_jump_unit {
    SRNG_JUMP_DRAWS = 0,       /* n draws                      */
    SRNG_JUMP_SUBSTREAMS = 1,  /* n * 2^76 draws (MRG32k3a)    */
    SRNG_JUMP_STREAMS = 2      /* n * 2^127 draws (MRG32k3a)   */
} srng_jump_unit;

typedef struct srng_set srng_set;

/* Launch shape of the generation kernels.  Any zero field takes the
 * library's default (or the value set by srng_set_tune).  Values never change
 * the output, only the speed.
 *   block_threads : threads per block (multiple of 32, 32..1024)
 *   blocks_per_sm : resident blocks per SM the grid is sized for (grid =
 *                   SM count x blocks_per_sm, work taken by grid stride)
 *   chunk         : MRG32k3a draws per thread item (a stream longer than this
 *                   is split into chunks whose start states are reached by
 *                   jump-ahead); multiple of 32
 *   unroll        : Philox blocks per thread per loop trip (1, 2 or 4)
 *   vector_store  : 1 = wide (16/32-byte) stores where the output alignment
 *                   allows, staged through shared memory so each warp store
 *                   covers whole 128-byte lines; 2 = never (element stores,
 *                   always coalesced); 3 = MRG32k3a whole-chunk rows written
 *                   by each lane directly with 32-byte stores (one full
 *                   sector per lane), else as 1; 4 = as 3, and for MRG32k3a
 *                   FP64 output three of every eight doubles (the 1st, 5th
 *                   and 7th) are the FP64 multiply z * norm itself while the
 *                   rest are built from integers (the same bits), so the FP64
 *                   unit shares the conversion work.  Default: 1 for the counter-based
 *                   generators and TinyMT32; for MRG32k3a 4 for FP64, and
 *                   for 4-byte values 3 when every stream of the call is cut
 *                   into a multiple of 32 chunks, else 1
 *   lane_blocks   : batched launches only: Philox blocks each lane computes
 *                   per work item (a Philox work item covers 32 x lane_blocks
 *                   blocks of one instance); MRG32k3a work items are 32
 *                   chunks of `chunk` draws of one instance
 *   resident      : MRG32k3a generation: at most this many blocks resident on
 *                   an SM at once, held by reserving shared memory (0: the
 *                   default, 6 for FP64 output and no limit otherwise; 32: as
 *                   many as the kernel's registers allow)                     */
typedef struct srng_tune {
    uint32_t block_threads;
    uint32_t blocks_per_sm;
    uint32_t chunk;
    uint32_t unroll;
    uint32_t vector_store;
    uint32_t lane_blocks;
    uint32_t resident;
    uint32_t reserved;
} srng_tune;

/* ------------------------------------------------------------------ errors */

/* Message of the last failed call on this host thread ("" if none). */
const char *srng_last_error(void);
/* Static name of a status code. */
const char *srng_status_string(srng_status status);
/* SRNG_ABI_VERSION of the loaded library. */
int srng_abi_version(void);

/* ---------------------------------------------------------- stream sets */

/* Create a set of n_streams streams of generator `gen` (paper Sec. 5.1: one
 * host call places every stream before any kernel runs).
 *   MRG32k3a: the seed is expanded into the six state words by SplitMix64
 *     (Steele, Lea & Flood 2014): six successive outputs r0..r5 give
 *     x1[i] = r_i mod m1, x2[i] = r_(i+3) mod m2, an all-zero component being
 *     replaced by (12345, 12345, 12345).  Stream i starts at A^(i * 2^e) y0
 *     with e = 127 (SRNG_SPACING_STREAM) or 76 (SRNG_SPACING_SUBSTREAM); the
 *     start states are computed on the device by the jump-ahead kernel.
 *   Philox4x32-10: key = (seed & 0xffffffff, seed >> 32); stream s uses
 *     counter words 2-3 = s and counter words 0-1 = position / 4, draw =
 *     word position % 4; every position starts at 0.  `spacing` is ignored.
 *   Philox4x32-10, keyed (SRNG_PHILOX4X32_10_KEYED; the paper's Sec. 4.3
 *     parameterisation: the key is the stream's own identifier): stream s
 *     uses key = (s & 0xffffffff, s >> 32), counter words 2-3 = the seed's
 *     two words, counter words 0-1 = position / 4.  Everything else as
 *     above; srng_describe reports this generator value.
 *   Threefry4x32-20 (SRNG_THREEFRY4X32_20; Salmon et al. 2011, named in the
 *     paper's Sec. 4.3 beside Philox, key per stream): stream s uses the
 *     128-bit key (s & 0xffffffff, s >> 32, seed & 0xffffffff, seed >> 32)
 *     and counter (position / 4 low, high, 0, 0), draw = word position % 4;
 *     conversions, positions and limits as Philox.  Tuning entries are
 *     shared with Philox (srng_set_tune of either applies to both).
 *   Threefry4x64-20 (SRNG_THREEFRY4X64_20; the 64-bit-word form): stream s
 *     uses key (s, seed, 0, 0) and counter (position / 8, 0, 0, 0) as 64-bit
 *     words; a block gives eight 32-bit draws, the low then the high half of
 *     each word, draw = 32-bit word position % 8.  Otherwise as Threefry4x32.
 * n_streams: 1 .. 2^40 (MRG32k3a with SRNG_SPACING_STREAM: at most 2^64 by
 * the paper, here limited by device memory: 48 bytes per stream, the working
 * states and the start states srng_reset restores; Philox and Threefry: 8).
 * The set owns its device memory until srng_destroy.  Synchronises
 * cuda_stream before returning (the set is ready to use on any stream). */
srng_status srng_create(srng_set **out, srng_gen gen, uint64_t seed, uint64_t n_streams,
                        srng_spacing spacing, void *cuda_stream);

/* Same, MRG32k3a only, from an explicit seed state y0 = (x1[n-3], x1[n-2],
 * x1[n-1], x2[n-3], x2[n-2], x2[n-1]).  SRNG_ERR_STATE unless every x1 word
 * is < m1, every x2 word < m2 and neither component is all zero. */
srng_status srng_create_from_state(srng_set **out, const uint32_t state[6], uint64_t n_streams,
                                   srng_spacing spacing, void *cuda_stream);

/* A set holding streams [stream_base, stream_base + n_streams) of the same
 * sequence (the set's stream i is stream stream_base + i of srng_create's
 * numbering; every stream-index argument of the other calls is relative to
 * the set): replicas on several GPUs each hold their own range, and stream
 * numbers up to 2^64 - 1 (the paper's 2^64 streams, Sec. 4.1) are reachable
 * without allocating the streams below them.  `state` NULL: from `seed` as
 * srng_create; else MRG32k3a from an explicit seed state (as
 * srng_create_from_state; `seed` ignored).  SRNG_ERR_RANGE if
 * stream_base + n_streams - 1 passes 2^64 - 1. */
srng_status srng_create_range(srng_set **out, srng_gen gen, uint64_t seed, const uint32_t state[6],
                              uint64_t stream_base, uint64_t n_streams, srng_spacing spacing, void *cuda_stream);

/* TinyMT32 (paper Sec. 4.2; Saito & Matsumoto 2011).  A 127-bit GF(2)-linear
 * state of four uint32 words (bit 31 of word 0 unused) and a parameter set
 * (mat1, mat2, tmat).  One step:
 *   x = (s0 & 0x7fffffff) ^ s1 ^ s2;  x ^= x << 1;  y = s3 ^ (s3 >> 1) ^ x;
 *   (s0, s1, s2, s3) = (s1, s2, x ^ (y << 10), y);  if y is odd: s1 ^= mat1,
 *   s2 ^= mat2.
 * Draw = tempering of the stepped state: t = s0 + (s2 >> 8);
 *   v = s3 ^ t, and ^ tmat when t is odd.  Conversions as Philox (32-bit words).
 * The paper's hybrid partition: the n_params parameter sets each serve a group
 * of group_size consecutive streams (a CUDA block's threads); stream j of a
 * group starts j * 2^64 steps after the group's seed state (sequence
 * splitting; the period is 2^127 - 1).  The seed state of a group is the
 * TinyMT32 seeding of (seed mod 2^32) with the group's parameters (words
 * (seed, mat1, mat2, tmat), seven mixing steps w ^= i + 1812433253 (p ^ (p >> 30)),
 * an all-zero state replaced, eight steps).
 *
 * srng_create_tinymt: params = 3 uint32 per set (mat1, mat2, tmat); every set
 *   must have period 2^127 - 1 (SRNG_ERR_ARG otherwise); n_streams =
 *   n_params * group_size (<= 2^40).  Synchronises cuda_stream.
 * srng_create(SRNG_TINYMT32, seed, n_streams, ...) = srng_create_tinymt with
 *   group_size 256 and ceil(n_streams / 256) parameter sets found by
 *   srng_tinymt_find_params(seed, ...); the last group may be partial.
 * srng_tinymt_find_params: parameter sets with period 2^127 - 1 drawn in
 *   order from SplitMix64(seed) (two outputs a, b per candidate: mat1 = a mod
 *   2^32, mat2 = a >> 32, tmat = b mod 2^32; a candidate is kept when the
 *   characteristic polynomial of the step, found by Berlekamp-Massey, has
 *   degree 127 and is irreducible -- primitive, 2^127 - 1 being prime).  The
 *   tempering parameter is not tuned for equidistribution.  Host only;
 *   about 1-2 ms per set, spread over the host's cores.
 * srng_tinymt_check_params: *max_period = 1 when (mat1, mat2) gives period
 *   2^127 - 1.
 * Jumps (srng_jump, SRNG_JUMP_DRAWS only) and chunked generation use
 * T^J s = r(T) s with r = x^J mod p: the polynomial on the host, its
 * evaluation on each state (Horner's rule, 127 steps) on the device.
 * TinyMT sets are not accepted by the batch calls or the server
 * (SRNG_ERR_UNSUPPORTED). */
srng_status srng_create_tinymt(srng_set **out, const uint32_t *params, uint64_t n_params, uint64_t group_size,
                               uint64_t seed, void *cuda_stream);
srng_status srng_tinymt_find_params(uint64_t seed, uint32_t count, uint32_t *params_out);
srng_status srng_tinymt_check_params(uint32_t mat1, uint32_t mat2, int *max_period);

/* Free the set and its device memory (after the device is done with it:
 * synchronises the device first).  NULL is accepted. */
srng_status srng_destroy(srng_set *set);

/* Put every stream of the set back at its start: MRG32k3a and TinyMT32 sets
 * copy back the start states placed at creation (a copy of the states is
 * kept for this: 24 or 16 bytes per stream), counter-based sets zero their
 * positions. */
srng_status srng_reset(srng_set *set, void *cuda_stream);

/* Description of a set. */
typedef struct srng_set_desc {
    srng_gen gen;
    srng_spacing spacing;
    uint64_t n_streams;
    uint64_t seed;
    uint32_t seed_state[6]; /* MRG32k3a y0; Philox: seed words in [0], [1] */
    uint64_t stream_base;   /* stream number of the set's first stream     */
} srng_set_desc;
srng_status srng_describe(const srng_set *set, srng_set_desc *out);

/* Move streams [stream_begin, stream_begin + count) forward by
 * n = n_hi * 2^64 + n_lo units (paper Sec. 2.3 sequence splitting).
 *   MRG32k3a: state <- A^(n * 2^u) state, u = 0, 76 or 127 by `unit`; the
 *     3x3 power is computed exactly on the host, its product with each state
 *     on the device.
 *   Philox: only SRNG_JUMP_DRAWS with n_hi = 0; position += n_lo
 *     (SRNG_ERR_RANGE if a position would pass 2^64 - 1).
 *   TinyMT32: only SRNG_JUMP_DRAWS; state <- T^n state (any 128-bit n).  */
srng_status srng_jump(srng_set *set, uint64_t stream_begin, uint64_t count, srng_jump_unit unit,
                      uint64_t n_hi, uint64_t n_lo, void *cuda_stream);

/* Generate n_per_stream values of type `type` from each of streams
 * [stream_begin, stream_begin + stream_count) into out_dev (stream-major, see
 * above; needs stream_count * n_per_stream * sizeof(type) bytes, any
 * alignment of the element size; 16-byte alignment is fastest) and move the
 * streams forward by n_per_stream draws.  Asynchronous on cuda_stream.
 * MRG32k3a: the call's state advance is launched as a programmatic dependent
 * of its generation kernel (scheduled while the last blocks run, it waits for
 * the kernel to finish); the advance itself allows no early launch, so work
 * the caller enqueues after the call starts only when both have finished. */
srng_status srng_generate(srng_set *set, uint64_t stream_begin, uint64_t stream_count,
                          uint64_t n_per_stream, srng_out type, void *out_dev, void *cuda_stream);

/* Same, with an explicit launch shape (NULL = defaults).  Output identical. */
srng_status srng_generate_tuned(srng_set *set, uint64_t stream_begin, uint64_t stream_count,
                                uint64_t n_per_stream, srng_out type, void *out_dev,
                                const srng_tune *tune, void *cuda_stream);

/* Same result as srng_generate, written to a HOST buffer.  Pinned host
 * memory that the device can address (cudaHostAlloc, cudaHostRegister) is
 * written directly by the generation kernels over the host link.  Other
 * (pageable) memory goes through an internal device staging ring (allocated
 * on first use, kept by the set, 2 x 256 MiB) whose pieces are copied to the
 * host while the next piece is generated.  Synchronises cuda_stream before
 * returning. */
srng_status srng_generate_host(srng_set *set, uint64_t stream_begin, uint64_t stream_count,
                               uint64_t n_per_stream, srng_out type, void *out_host,
                               void *cuda_stream);

/* Copy per-stream state to / from the host (checkpoint / resume; paper
 * Sec. 1 asks for reproducible streams).  MRG32k3a: 6 uint32 per stream in
 * the order of srng_create_from_state; Philox and Threefry: one uint64
 * position per stream; TinyMT32: 4 uint32 per stream (s0..s3).
 * srng_set_state validates MRG32k3a states (SRNG_ERR_STATE) and rejects
 * all-zero TinyMT32 states (bit 31 of s0 ignored).
 * Both synchronise cuda_stream. */
srng_status srng_get_state(const srng_set *set, uint64_t stream_begin, uint64_t count,
                           void *state_host, void *cuda_stream);
srng_status srng_set_state(srng_set *set, uint64_t stream_begin, uint64_t count,
                           const void *state_host, void *cuda_stream);

/* Default launch shape used by srng_generate for (gen, type); NULL resets
 * it to the built-in default.  Process-wide. */
srng_status srng_set_tune(srng_gen gen, srng_out type, const srng_tune *tune);
srng_status srng_get_tune(srng_gen gen, srng_out type, srng_tune *out);

/* Integer -> uniform conversion alone: out_dev[i] = convert(in_dev[i]) with
 * the generator's fixed rule for `type` (see the header comment).  For
 * SRNG_MRG32K3A the inputs must be combined values in [1, m1]
 * (SRNG_OUT_F64 assumes it; other values give the same formula's result). */
srng_status srng_convert(srng_gen gen, srng_out type, const uint32_t *in_dev, uint64_t n,
                         void *out_dev, void *cuda_stream);

/* Device view of a set for use inside user kernels with srng_device.cuh
 * (the paper's in-kernel constructor + next(), Sec. 5.2).  The pointers stay
 * owned by the set and valid until srng_destroy. */
typedef struct srng_dev_view {
    int32_t gen;            /* SRNG_MRG32K3A, SRNG_PHILOX4X32_10 (either layout),
                             * SRNG_THREEFRY4X32_20, SRNG_THREEFRY4X64_20 or
                             * SRNG_TINYMT32                                    */
    uint32_t key0, key1;    /* Philox / Threefry: the set's seed words (Philox
                             * key, or counter words 2-3 when keyed; Threefry4x32
                             * key words 2-3; Threefry4x64 key word 1)          */
    uint32_t flags;         /* bit 0: Philox keyed layout (key = stream)        */
    uint64_t n_streams;
    uint32_t *mrg_state;    /* MRG32k3a, SoA: word j of stream i at
                             * [j * n_streams + i], j in the srng_create_from_state order */
    uint64_t *philox_pos;   /* Philox / Threefry: position of each stream       */
    uint64_t stream_base;   /* stream number of slot 0 (srng_create_range)      */
    uint32_t *tinymt_state; /* TinyMT32, SoA: word j of stream i at
                             * [j * n_streams + i]                              */
    const uint32_t *tinymt_params; /* TinyMT32: (mat1, mat2, tmat, 0) per set */
    uint64_t tinymt_group_size;    /* TinyMT32: streams per parameter set     */
} srng_dev_view;
srng_status srng_get_device_view(const srng_set *set, srng_dev_view *out);

/* Non-uniform variates from FP32 uniforms (SRNG_OUT_F32 outputs of either
 * generator; the paper itself covers uniforms only).
 *   SRNG_DIST_EXPONENTIAL: out[i] = -ln(1 - in[i]), rate 1;
 *   SRNG_DIST_NORMAL: Box-Muller on the pairs (in[2k], in[2k+1]):
 *     r = sqrt(-2 ln(1 - in[2k])), t = 2 pi in[2k+1],
 *     out[2k] = r cos t, out[2k+1] = r sin t (n must be even).
 * ln, sin and cos are this library's own (srng_device.cuh, srng::dist), every
 * step one correctly rounded IEEE single operation or fused multiply-add, so
 * the results are reproducible bit for bit on any IEEE machine that follows
 * the same steps; in and out may be the same buffer.  Inputs must lie in
 * [0, 1).  Asynchronous on cuda_stream. */
typedef enum srng_dist {
    SRNG_DIST_EXPONENTIAL = 0,
    SRNG_DIST_NORMAL = 1
} srng_dist;
srng_status srng_transform(srng_dist dist, const float *in_dev, uint64_t n, float *out_dev, void *cuda_stream);

/* ------------------------------------------------------------ host maths */

/* The SplitMix64 seed expansion used by srng_create (pure host function). */
srng_status srng_seed_expand(uint64_t seed, uint32_t state[6]);

/* The jump matrices A1^d mod m1 and A2^d mod m2, d = n * 2^u (u by `unit`),
 * row-major 3x3, acting on (x[n-3], x[n-2], x[n-1]).  Pure host function. */
srng_status srng_jump_matrix(srng_jump_unit unit, uint64_t n_hi, uint64_t n_lo, uint32_t a1[9],
                             uint32_t a2[9]);

/* ----------------------------------------------- batched instances (K4/K5) */

/* One simulation instance of a batch: `length` draws of stream `stream` of
 * set sets[set_index], starting `offset` draws after that stream's current
 * position (the batch reads the set, it does not move it). */
typedef struct srng_instance {
    uint32_t set_index;
    uint32_t reserved;
    uint64_t stream;
    uint64_t offset;
    uint64_t length;
    uint64_t out_offset; /* element offset of the instance's output (WRITE mode) */
} srng_instance;

typedef enum srng_batch_mode {
    SRNG_BATCH_WRITE = 0,    /* write the values (type `type`) at out_offset            */
    SRNG_BATCH_FUSED_PI = 1  /* no values written: count, per instance, the pairs
                              * (draw 2k, draw 2k+1), k < length/2, inside the quarter
                              * disc, tested exactly on the uniforms (Philox:
                              * a^2 + b^2 < 2^48 with a = w >> 8; MRG32k3a:
                              * z0^2 + z1^2 < (m1+1)^2); int64 per instance          */
} srng_batch_mode;

typedef struct srng_batch_plan srng_batch_plan;

/* Build a batch plan: instance start states (jump-ahead kernel), the flat work
 * list (fixed-size chunks of every instance, mixed generators) and a CUDA
 * graph of {reset work counter, zero counts, persistent kernel}.  `out_dev`
 * is where launches write: WRITE mode -> values; FUSED_PI -> n_inst int64
 * counts.  The plan keeps pointers to `sets` (they must outlive it) but
 * copies `inst`.  Synchronises cuda_stream. */
srng_status srng_batch_plan_create(srng_batch_plan **out, srng_set *const *sets, uint32_t n_sets,
                                   const srng_instance *inst, uint64_t n_inst, srng_batch_mode mode,
                                   srng_out type, void *out_dev, const srng_tune *tune,
                                   void *cuda_stream);
/* Launch the captured graph once on cuda_stream (asynchronous). */
srng_status srng_batch_plan_launch(srng_batch_plan *plan, void *cuda_stream);
/* Number of kernel launches one srng_batch_plan_launch performs: one
 * persistent kernel per generator family present (MRG32k3a items; Philox and
 * Threefry items), both nodes of the one captured graph. */
srng_status srng_batch_plan_info(const srng_batch_plan *plan, uint64_t *n_work_items,
                                 uint32_t *kernels_per_launch);
srng_status srng_batch_plan_destroy(srng_batch_plan *plan);

/* One-shot batch: create a plan, launch it, wait, destroy it. */
srng_status srng_batch_run(srng_set *const *sets, uint32_t n_sets, const srng_instance *inst,
                           uint64_t n_inst, srng_batch_mode mode, srng_out type, void *out_dev,
                           void *cuda_stream);

/* --------------------------------------------------- serving loop (K6) */

/* A request server over one stream set (paper Sec. 2.1: every processing
 * element, here every request, autonomously gets its own part of its own
 * stream).  A native dispatcher thread keeps the set's states on the device,
 * admits submitted requests in arrival order as soon as their output fits in
 * the output pool (the memory budget), cuts admitted work into steps of at
 * most max_step_draws draws gathered across requests (continuous batching:
 * requests that arrive while steps run join the next step), and runs up to
 * max_inflight steps at once on separate CUDA streams with the batch kernel.
 *
 * Positions: a request for n draws of stream s receives the next n positions
 * of s, counted from the set's state when the server was created, reserved at
 * submission in submission order -- so every result depends only on the
 * sequence of submissions, never on how requests were batched.  The server
 * does not move the set; do not jump, reset, generate from or destroy the set
 * while the server exists. */
typedef struct srng_server srng_server;

typedef struct srng_server_config {
    uint64_t budget_bytes;      /* output pool allocated at create (0: 16 GiB)                 */
    uint32_t max_inflight;      /* steps on the device at once, 1..8 (0: 4)                    */
    uint32_t max_step_requests; /* request parts per step, 1..65536 (0: 4096)                  */
    uint64_t max_step_draws;    /* draws per step (0: 2^30); larger requests span steps        */
    uint32_t chunk;             /* MRG32k3a draws per lane chunk, multiple of 32 (0: by step:  */
                                /* 128 below 2^23 draws, 256 below 2^27, else 1024)            */
    uint32_t lane_blocks;       /* Philox blocks per lane per work item (0: 64)                */
    uint32_t reserved[4];
} srng_server_config;

typedef struct srng_server_stats {
    uint64_t submitted, completed, rejected;
    uint64_t draws_completed;
    uint64_t steps;             /* steps launched                                              */
    uint64_t kernels;           /* kernels launched: set-up, MRG32k3a item starts (one kernel  */
                                /* for both in a small MRG32k3a step), batch                   */
    double p50_us, p99_us;      /* latency, submission -> completion seen by the dispatcher    */
    double mean_us, max_us;
    double wall_s;              /* first submission -> last completion                         */
    uint64_t peak_pool_bytes;   /* largest pool use                                            */
} srng_server_stats;

/* Create a server over `set` (MRG32k3a or Philox).  cfg may be NULL
 * (defaults).  Allocates the pool and per-step buffers once. */
srng_status srng_server_create(srng_server **out, srng_set *set, const srng_server_config *cfg);
/* Submit a request for n draws of `stream` as `type`; non-blocking.  Returns
 * a ticket.  SRNG_ERR_BUDGET if n * sizeof(type) exceeds the whole pool;
 * SRNG_ERR_RANGE if the stream is outside the set. */
srng_status srng_server_submit(srng_server *srv, uint64_t stream, uint64_t n, srng_out type, uint64_t *ticket);
/* Same, at an explicit start position (no reservation): the draws
 * [pos, pos + n) of `stream`. */
srng_status srng_server_submit_at(srng_server *srv, uint64_t stream, uint64_t pos, uint64_t n, srng_out type,
                                  uint64_t *ticket);
/* done = 1 once the request's output is complete; out_dev (may be NULL) then
 * points to its n values inside the pool, valid until srng_server_release. */
srng_status srng_server_poll(srng_server *srv, uint64_t ticket, int *done, const void **out_dev);
/* Block until done or timeout_ms passes (SRNG_ERR_TIMEOUT; the request stays
 * queued or running). */
srng_status srng_server_wait(srng_server *srv, uint64_t ticket, uint32_t timeout_ms, const void **out_dev);
/* Give the request's output memory back to the pool (after completion);
 * SRNG_ERR_CLOSED for an unknown ticket, SRNG_ERR_ARG if not yet complete. */
srng_status srng_server_release(srng_server *srv, uint64_t ticket);
/* Copy a completed request's n values to dst (host memory if dst_is_host,
 * else device memory); synchronous.  SRNG_ERR_ARG if not yet complete. */
srng_status srng_server_read(srng_server *srv, uint64_t ticket, void *dst, int dst_is_host);
srng_status srng_server_get_stats(srng_server *srv, srng_server_stats *out);
srng_status srng_server_reset_stats(srng_server *srv);
/* Stop the dispatcher (finishing the steps on the device), free everything. */
srng_status srng_server_destroy(srng_server *srv);

/* One request of a trace: arrival time (seconds after the replay starts). */
typedef struct srng_request {
    double arrival_s;
    uint64_t stream;
    uint64_t n;
} srng_request;

/* Replay a trace on the server from a native client thread: each request is
 * submitted at its arrival time (or at once when time_scale = 0) and its
 * output released as soon as it completes; returns when all have completed
 * (or SRNG_ERR_TIMEOUT after timeout_ms).  Statistics cover this replay. */
srng_status srng_server_replay(srng_server *srv, const srng_request *req, uint64_t n_req, srng_out type,
                               double time_scale, uint32_t timeout_ms, srng_server_stats *out);

/* ------------------------------------------- batched, without allocating */

/* The paper has no counterpart to this entry point.  It gives the result of
 * srng_batch_run to callers that must not allocate device memory per call:
 * code whose device memory belongs to another allocator (a framework's
 * caching allocator that holds the GPU, a plugin host that forbids
 * cudaMalloc) and latency-critical loops that cannot pay for cudaMalloc /
 * cudaFree and the device synchronisation cudaFree brings.
 *
 * Same arguments, same output, bit for bit, as srng_batch_run.  On success the
 * call allocates nothing, on the host or on the device: its scratch (instance
 * descriptors, per-instance work-item counts, the work counter) is one
 * fixed-size __device__ array of about 0.6 MB inside this library, which
 * every GPU that loads the library holds until the process exits.  Limits:
 * at most SRNG_BATCH_STATIC_MAX_INSTANCES instances and
 * SRNG_BATCH_STATIC_MAX_SETS sets, MRG32k3a instances of at most 2^41 draws
 * and at most 2^31 work items in one call (an MRG32k3a item covers up to
 * 16,384 draws, a counter-based one up to 8,192; the kernels count items in
 * 32-bit words), else SRNG_ERR_ARG with nothing enqueued.
 *
 * The first call on a device does that device's set-up (it looks up the
 * array's device address with cudaGetSymbolAddress and sizes the grid); make
 * that first call before any stream capture.  The call is asynchronous on
 * cuda_stream: it copies `inst` to the device with cudaMemcpyAsync on that
 * stream, then launches three kernels (descriptors, prefix
 * sums with the zeroing of the work counter and of the FUSED_PI counts, the
 * persistent batch kernel).  Every call shares the one array, which keeps the
 * last call's contents: calls whose work overlaps on the GPU (different
 * streams without ordering, or several host threads on different streams)
 * race on it.  Order the calls on one stream, or synchronise between them.
 * When `inst` is pageable host memory the runtime stages the copy before the
 * call returns, so the caller may reuse `inst` at once.  When it is
 * page-locked host memory the copy runs later, in stream order: keep `inst`
 * unchanged until the stream has passed the call (for instance, until
 * cudaStreamSynchronize or an event recorded after it). */
#define SRNG_BATCH_STATIC_MAX_INSTANCES 4096
#define SRNG_BATCH_STATIC_MAX_SETS 8
srng_status srng_batch_run_static(srng_set *const *sets, uint32_t n_sets, const srng_instance *inst,
                                  uint64_t n_inst, srng_batch_mode mode, srng_out type, void *out_dev,
                                  void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SRNG_H */
