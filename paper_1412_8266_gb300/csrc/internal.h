// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "srng.h"

namespace srng_impl {

// Element type of each output type (the fused variates are FP32).
template <int OUT> struct OutType;
template <> struct OutType<SRNG_OUT_U32> { using T = uint32_t; };
template <> struct OutType<SRNG_OUT_F32> { using T = float; };
template <> struct OutType<SRNG_OUT_F64> { using T = double; };
template <> struct OutType<SRNG_OUT_EXP_F32> { using T = float; };
template <> struct OutType<SRNG_OUT_NORMAL_F32> { using T = float; };

// ------------------------------------------------------------------ errors
// Record a failure message for srng_last_error() and return the status.
srng_status fail(srng_status st, const std::string &msg);
// Map a CUDA error to SRNG_ERR_CUDA (or SRNG_ERR_OOM) with context.
srng_status cuda_fail(cudaError_t e, const char *what);
void clear_error();

#define SRNG_CUDA_TRY(expr)                                          \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return ::srng_impl::cuda_fail(_e, #expr); \
    } while (0)

// ------------------------------------------------------------- host maths
constexpr uint64_t kM1 = 4294967087ull;
constexpr uint64_t kM2 = 4294944443ull;

// 3x3 matrices mod m (row-major, entries < m) for both components.
struct MatPair {
    uint32_t a[18];  // [0..8] component 1 (mod m1), [9..17] component 2 (mod m2)
};

MatPair mat_identity();
MatPair mat_mul(const MatPair &x, const MatPair &y);
// A^d with d = n * 2^shift, n = (hi, lo) 128-bit; shift in [0, 127].
MatPair mat_pow_shifted(uint64_t n_hi, uint64_t n_lo, int shift);
// A^(2^k) for k in [0, 255].
MatPair mat_pow2(int k);
void seed_expand(uint64_t seed, uint32_t out[6]);
bool state_valid(const uint32_t s[6]);

// -------------------------------------------------------------- devices
struct DeviceInfo {
    int device;
    int sm_count;
};
srng_status current_device(DeviceInfo *out);

// The kernels (and tuning tables) of a generator value: the keyed Philox
// layout runs the Philox kernels.
inline int kernel_gen(int g)
{
    return g == SRNG_MRG32K3A ? SRNG_MRG32K3A : g == SRNG_TINYMT32 ? SRNG_TINYMT32 : SRNG_PHILOX4X32_10;
}
// Row of the tuning tables of a kernel family.
inline int tune_row(int g) { return g == SRNG_MRG32K3A ? 0 : g == SRNG_TINYMT32 ? 2 : 1; }

// ---------------------------------------------------------------- tuning
srng_tune effective_tune(srng_gen gen, srng_out type, const srng_tune *user);
srng_status check_tune(const srng_tune *t);

// --------------------------------------------------------- jump tables
// Up to 64 matrix pairs J_k = B^(2^k) for a base matrix pair B; applied for
// each set bit of an index (start of stream/chunk = B^index y).
struct JumpTable {
    uint32_t m[64][18];
};

// Radix-32 chunk starts: lane[l] = A^(C l) and warp[g] = A^(32 C g), l, g < 32,
// for chunks of C draws (both components, 18 words each).
struct RadixTable {
    uint32_t lane[32][18];
    uint32_t warp[32][18];
};

// ------------------------------------------------------------ kernels
// K1: stream placement and jumps (jump.cu).
// Slots [first, first + count) get streams index_base + slot: y0 times J_k for
// every set bit k of the stream number.
cudaError_t launch_mrg_place(uint32_t *state, uint64_t n_streams, uint64_t first, uint64_t count,
                             uint64_t index_base, const uint32_t y0[6], const JumpTable &tab, int nbits,
                             cudaStream_t stream, const DeviceInfo &dev);
// dependent: launched right after an MRG32k3a generation kernel on the same
// stream, as its programmatic dependent (scheduled early, waits for it).
cudaError_t launch_mrg_apply(uint32_t *state, uint64_t n_streams, uint64_t first, uint64_t count,
                             const MatPair &m, cudaStream_t stream, const DeviceInfo &dev,
                             bool dependent = false);
cudaError_t launch_philox_advance(uint64_t *pos, uint64_t first, uint64_t count, uint64_t n,
                                  cudaStream_t stream, const DeviceInfo &dev);

// K2 / K3 / conversion (generate.cu).
struct MrgGenArgs {
    const uint32_t *state;
    uint64_t n_streams;   // SoA stride
    uint64_t s_begin, s_count, n;
    uint64_t chunk;       // draws per thread item
    uint64_t cps;         // chunks per stream
    int nbits;            // table entries used for the chunk jumps
    void *out;
};
// rt: radix-32 chunk starts (used by the direct-row kernels when the chunk
// count per stream is a multiple of 32), or null.
cudaError_t launch_mrg_generate(const MrgGenArgs &a, srng_out type, const JumpTable &tab,
                                const srng_tune &t, cudaStream_t stream, const DeviceInfo &dev,
                                const RadixTable *rt = nullptr);

struct PhiloxGenArgs {
    uint64_t stream_base; // stream number of the set's slot 0
    uint32_t k0, k1;      // the set's seed words
    int keyed;            // 0: key = (k0, k1), counter words 2-3 = stream; 1: key = stream, words 2-3 = (k0, k1)
    int threefry;         // 1: Threefry4x32-20, key = (stream, k0, k1), counter words 2-3 = 0;
                          // 2: Threefry4x64-20, 64-bit key = (stream, k1:k0, 0, 0)
    const uint64_t *pos;
    uint64_t s_begin, s_count, n;
    void *out;
};
cudaError_t launch_philox_generate(const PhiloxGenArgs &a, srng_out type, const srng_tune &t,
                                   cudaStream_t stream, const DeviceInfo &dev);

cudaError_t launch_convert(srng_gen gen, srng_out type, const uint32_t *in, uint64_t n, void *out,
                           cudaStream_t stream, const DeviceInfo &dev);
cudaError_t launch_transform(int dist, const float *in, uint64_t n, float *out, cudaStream_t stream,
                             const DeviceInfo &dev);

// ------------------------------------------------- batched work (batch.cu)
// Per-instance descriptor on the device.
struct BatchInst {
    uint32_t gen;             // SRNG_MRG32K3A, SRNG_PHILOX4X32_10 or SRNG_THREEFRY4X32_20
    uint32_t key0, key1;      // Philox key of this instance's stream (Threefry: key words 0-1)
    uint32_t st[6];           // MRG32k3a start state (written by the set-up kernel)
    uint64_t stream;          // stream index in its set
    uint64_t ctr_hi;          // Philox counter words 2-3 (the stream, or the seed when keyed);
                              // Threefry key words 2-3 (the seed)
    uint64_t offset;          // draws after the stream's current position
    uint64_t pos;             // Philox start position (written by the set-up kernel)
    uint64_t length;
    uint64_t out_offset;
    const uint32_t *src_state;  // MRG32k3a set states (SoA) and their stride
    uint64_t src_ns;
    const uint64_t *src_pos;    // Philox set positions
};

struct BatchArgs {
    const BatchInst *inst;
    const uint2 *items;       // {instance, first chunk (MRG32k3a) or segment (Philox)}
    uint32_t *counter;
    uint64_t n_items;
    uint64_t chunk;           // MRG32k3a draws per lane-chunk
    uint32_t lane_blocks;     // Philox blocks per lane per item
    int32_t mode;             // srng_batch_mode
    void *out;                // values (WRITE) or int64 counts (FUSED_PI)
    // MRG32k3a items, optional: the state at each item's first chunk (6 words
    // per item, in item order) and the lane table A^(chunk l), l < 32 (18 words
    // each); when set, lane l starts from its item's state with one jump.
    const uint32_t *item_state;
    const uint32_t *lane_tab;
};

// Launchers shared by the batch plan and the server.
// Instance start states: MRG32k3a = A^offset applied to the stream state;
// Philox = stream position + offset (reads src_* fields, writes st / pos).
// zero: a work counter the kernel sets to 0 (or null)
cudaError_t launch_batch_setup(BatchInst *d_inst, uint64_t n, cudaStream_t s, uint32_t *zero = nullptr);
// The persistent batch kernel over a.n_items items, all MRG32k3a (mrg) or all
// counter-based (!mrg); a.counter must be zero.
// Work-item families of the batch kernels: each kernel holds code for one.
enum BatchFamily { kBatchMrg = 0, kBatchCounter = 1, kBatchPhilox = 2 };  // counter: Philox and Threefry
cudaError_t launch_batch(const BatchArgs &a, srng_out type, BatchFamily fam, const JumpTable &chunk_tab, unsigned grid,
                         cudaStream_t s);
// State at the first chunk of every MRG32k3a item (the instance's start state
// moved by chunk_tab's J_k for the set bits of the item's first chunk):
// item_state[6 i + j], items[0, n) all MRG32k3a.
cudaError_t launch_batch_item_states(const BatchInst *d_inst, const uint2 *d_items, uint64_t n,
                                     const JumpTable &chunk_tab, uint32_t *item_state, cudaStream_t s);
// The same from the stream states directly (no set-up kernel needed before it);
// zero: the step's work counter, set to 0.
cudaError_t launch_batch_item_states_direct(const BatchInst *d_inst, const uint2 *d_items, uint64_t n,
                                            const JumpTable &chunk_tab, uint32_t *item_state, uint32_t *zero,
                                            cudaStream_t s);
// Lane table of the chunk size: A^(chunk l), l < 32, 18 words each (host).
void lane_jump_table(uint64_t chunk, uint32_t out[32 * 18]);
// Resident blocks per SM of the batch kernel for `type`.
int batch_blocks_per_sm(srng_out type, BatchFamily fam);
// The batch kernel family of a set's work items.
inline BatchFamily batch_family(const srng_set *s);
// J_k = A^(chunk 2^k), k < 64.
void chunk_jump_table(uint64_t chunk, JumpTable *out);
constexpr int kBatchThreads = 256;

// ------------------------------------------------ TinyMT32 (tinymt.cu, tinymt_host.cpp)
typedef unsigned __int128 u128;
// Seed state of a parameter set from a 32-bit seed (the TinyMT32 seeding).
void tmt_seed_state(uint32_t seed32, uint32_t mat1, uint32_t mat2, uint32_t tmat, uint32_t s[4]);
// True when (mat1, mat2) has period 2^127 - 1; *charpoly = the step's
// characteristic polynomial (degree 127).
bool tmt_max_period(uint32_t mat1, uint32_t mat2, u128 *charpoly);
// x^(e_hi 2^64 + e_lo) mod p.
u128 tmt_xpow(u128 p, uint64_t e_hi, uint64_t e_lo);
// a^2 mod p.
u128 tmt_square_mod(u128 p, u128 a);
// `count` parameter sets (mat1, mat2, tmat) from SplitMix64(seed), with
// their characteristic polynomials when polys is not NULL.
void tmt_find_params(uint64_t seed, uint32_t count, uint32_t *out, u128 *polys);

inline uint4 poly_words(u128 r)
{
    return make_uint4((uint32_t)r, (uint32_t)(r >> 32), (uint32_t)(r >> 64), (uint32_t)(r >> 96));
}

struct TmtGenArgs {
    uint32_t *state;           // SoA 4 x n_streams
    uint64_t n_streams;
    const uint4 *params;       // (mat1, mat2, tmat, 0) per group
    uint64_t group_size;
    uint64_t s_begin, s_count, n;
    uint64_t chunk, cps;       // draws per item, items per stream
    int nbits;                 // bits of the chunk index
    const uint4 *jtab;         // [group - g0][k] = x^(chunk 2^k) mod p_group, k < nbits
    uint64_t g0;
    int write_back;            // 1: one item per stream, its thread stores the advanced state
    void *out;
};
// Stream placement: stream i of group g = T^(j 2^64) seed[g], j = i - g group_size,
// jt[g][k] = x^(2^(64 + k)) mod p_g, k < nbits.
cudaError_t launch_tmt_place(uint32_t *state, uint64_t n_streams, const uint4 *params, uint64_t group_size,
                             const uint4 *seed_states, const uint4 *jt, int nbits, cudaStream_t stream,
                             const DeviceInfo &dev);
// state <- poly[group - g0](T) state for streams [first, first + count).
cudaError_t launch_tmt_apply(uint32_t *state, uint64_t n_streams, const uint4 *params, uint64_t group_size,
                             uint64_t first, uint64_t count, const uint4 *poly, uint64_t g0, cudaStream_t stream,
                             const DeviceInfo &dev);
cudaError_t launch_tmt_generate(const TmtGenArgs &a, srng_out type, const srng_tune &t, cudaStream_t stream,
                                const DeviceInfo &dev);

}  // namespace srng_impl

// The stream set object behind the opaque srng_set handle.
struct srng_set {
    srng_gen gen;
    srng_spacing spacing;
    uint64_t n_streams;
    uint64_t stream_base;    // stream number of slot 0 (a set may hold any range of streams)
    uint64_t seed;
    uint32_t y0[6];          // MRG32k3a seed state
    uint32_t key0, key1;     // Philox / Threefry seed words (Philox key, or counter words 2-3 when keyed)
    bool keyed;              // key = the stream (keyed Philox, Threefry)
    bool threefry;           // Threefry (counter-based family, kernels as Philox)
    bool threefry64;         // the Threefry4x64-20 form
    // TinyMT32: states, parameter sets and their characteristic polynomials
    uint64_t tmt_group_size = 0, tmt_n_groups = 0;
    uint32_t tmt_seed32 = 0;
    uint32_t *d_tstate = nullptr;            // SoA 4 x n_streams
    uint4 *d_tparams = nullptr;              // (mat1, mat2, tmat, 0) per group
    std::vector<uint32_t> tmt_params;        // host copy, 3 per group
    std::vector<srng_impl::u128> tmt_poly;   // per group
    // device polynomial tables by (kind, exponent words, first group, groups, bits);
    // kept until destroy (at most a few dozen) so no launch in flight loses its table
    std::map<std::array<uint64_t, 6>, uint4 *> tmt_tables;
    std::mutex tmt_mu;
    int device;
    uint32_t *d_state;       // MRG32k3a SoA states (6 x n_streams)
    uint32_t *d_start;       // the placed start states of d_state or d_tstate (srng_reset copies them back)
    size_t start_bytes;
    uint64_t *d_pos;         // Philox positions
    uint64_t max_pos;        // host-side upper bound on any Philox position
    // staging for srng_generate_host
    void *d_stage[2];
    size_t stage_bytes;
    cudaStream_t copy_stream;
    cudaEvent_t ev_gen[2], ev_copy[2];
    std::mutex mu;
};

namespace srng_impl {
// Generator value of a set's work descriptors: the kernels' choice of block function.
inline BatchFamily batch_family(const srng_set *s)
{
    return s->gen == SRNG_MRG32K3A ? kBatchMrg : s->threefry ? kBatchCounter : kBatchPhilox;
}

inline uint32_t inst_gen(const srng_set *s)
{
    return s->threefry64 ? SRNG_THREEFRY4X64_20 : s->threefry ? SRNG_THREEFRY4X32_20 : (uint32_t)s->gen;
}
}  // namespace srng_impl

