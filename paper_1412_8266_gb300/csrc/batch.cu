// K4 / K5 -- batched instances in one persistent, graph-captured launch.
//
// Thousands of simulation instances, each with its own stream (paper Sec. 4.1
// / 4.3: one stream per processing element) and its own length, mixed
// MRG32k3a and Philox4x32-10, are cut into equal-sized work items:
//   - MRG32k3a item: 32 consecutive chunks of `chunk` draws of one instance,
//     one chunk per lane; a lane reaches its chunk's start by jump-ahead
//     ((A^chunk)^t applied to the instance's start state, Sec. 2.3);
//   - Philox / Threefry item: 32 x lane_blocks consecutive 4-word counter
//     groups of one instance.
// A persistent grid (one wave of resident blocks) takes items from a global
// counter with one atomicAdd per warp and item, so instance lengths spread
// over five decades still load every SM evenly.  The plan captures, in one
// CUDA graph, {zero counters, zero counts} and one persistent kernel per
// generator family present (MRG32k3a items; counter-based items), the two
// kernels as independent graph nodes on a forked capture stream.
//
// Modes:
//   WRITE     values go to out[out_offset + k] (staged through shared memory
//             for MRG32k3a exactly as in the plain kernel);
//   FUSED_PI  nothing is written: draws stay in registers, pairs
//             (2k, 2k+1) are tested exactly against the quarter disc and the
//             per-lane counts are reduced (warp shuffle for counter-based
//             items, whose Threefry4x64 lanes take whole 8-word blocks; one
//             64-bit atomicAdd per lane-chunk for MRG32k3a items).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "counter_based.cuh"
#include "internal.h"
#include "srng_device.cuh"

namespace srng_impl {

namespace {

template <int GEN, int OUT>
__device__ __forceinline__ typename OutType<OUT>::T bconvert(uint32_t v)
{
    if constexpr (OUT == SRNG_OUT_U32) return v;
    else if constexpr (OUT == SRNG_OUT_F32) return srng::to_f32(v);
    else if constexpr (GEN == SRNG_MRG32K3A) return srng::mrg::to_f64(v);
    else return srng::philox::to_f64(v);
}

// Exact quarter-disc tests on the defined uniforms.
__device__ __forceinline__ uint32_t hit_mrg(uint32_t z0, uint32_t z1)
{
    // z0^2 + z1^2 < (m1 + 1)^2; the sum can pass 2^64, in which case it is a miss.
    const uint64_t a = (uint64_t)z0 * z0, s = a + (uint64_t)z1 * z1;
    const uint64_t r = (uint64_t)srng::mrg::kM1 + 1;
    return (s >= a && s < r * r) ? 1u : 0u;
}

__device__ __forceinline__ uint32_t hit_philox(uint32_t w0, uint32_t w1)
{
    const uint64_t a = w0 >> 8, b = w1 >> 8;
    return a * a + b * b < (1ull << 48) ? 1u : 0u;
}

constexpr int kWarps = 8;

template <int OUT>
struct Smem {
    using T = typename OutType<OUT>::T;
    static constexpr int G = 128 / sizeof(T);
    static constexpr int VPL = 16 / sizeof(T);
    static constexpr int RS = G + VPL;
    T tile[kWarps][32 * RS];
};

__device__ __forceinline__ void bst256(void *p, uint4 x, uint4 y)
{
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(x.x), "r"(x.y),
                 "r"(x.z), "r"(x.w), "r"(y.x), "r"(y.y), "r"(y.z), "r"(y.w)
                 : "memory");
}

// ---------------------------------------------------- MRG32k3a work item
// Lane l owns chunk t = first_chunk + l of the instance (chunk draws, the last
// chunk shorter).  Row r of the warp's tile is chunk first_chunk + r, which
// starts at element out_offset + (first_chunk + r) * chunk: rows are at a
// fixed stride, so row addresses and lengths are arithmetic.  32-byte stores
// (4 lanes per 128-byte row) when the instance's rows are 32-byte aligned,
// element stores (one row per warp instruction) otherwise.
template <int OUT>
__device__ void mrg_item(const BatchArgs &a, const JumpTable &tab, uint32_t it, uint32_t ii, uint32_t first_chunk,
                         Smem<OUT> &sm, int warp, int lane)
{
    using T = typename OutType<OUT>::T;
    constexpr int G = Smem<OUT>::G, VPL = Smem<OUT>::VPL, RS = Smem<OUT>::RS;
    constexpr int EPQ = 32 / sizeof(T);
    const BatchInst &in = a.inst[ii];
    const uint64_t t = (uint64_t)first_chunk + lane;
    const uint64_t start = t * a.chunk;
    const uint64_t len = start < in.length ? min(a.chunk, in.length - start) : 0;
    uint32_t s0, s1, s2, s3, s4, s5;
    if (a.item_state) {
        // the item's first-chunk state, then one jump by this lane's l chunks
        const uint32_t *is = a.item_state + 6 * (size_t)it;
        s0 = is[0]; s1 = is[1]; s2 = is[2]; s3 = is[3]; s4 = is[4]; s5 = is[5];
        if (len && lane) srng::mrg::jump(a.lane_tab + 18 * lane, s0, s1, s2, s3, s4, s5);
    } else {
        s0 = in.st[0]; s1 = in.st[1]; s2 = in.st[2]; s3 = in.st[3]; s4 = in.st[4]; s5 = in.st[5];
        if (len) {
            for (int k = 0; k < 40; ++k) {
                if ((t >> k) == 0) break;
                if ((t >> k) & 1) srng::mrg::jump(tab.m[k], s0, s1, s2, s3, s4, s5);
            }
        }
    }
    if (a.mode == SRNG_BATCH_FUSED_PI) {
        uint32_t hits = 0;
        for (uint64_t k = 0; k + 1 < len; k += 2) {
            const uint32_t z0 = srng::mrg::step(s0, s1, s2, s3, s4, s5);
            const uint32_t z1 = srng::mrg::step(s0, s1, s2, s3, s4, s5);
            hits += hit_mrg(z0, z1);
        }
        if (hits) atomicAdd(reinterpret_cast<unsigned long long *>(a.out) + ii, (unsigned long long)hits);
        return;
    }
    T *out = static_cast<T *>(a.out);
    T *my = &sm.tile[warp][lane * RS];
    const uint64_t row0 = in.out_offset + (uint64_t)first_chunk * a.chunk;  // row r starts at row0 + r * chunk
    const uint64_t first_start = (uint64_t)first_chunk * a.chunk;             // draw index of row 0
    const bool vec = ((reinterpret_cast<uintptr_t>(out + row0) & 31) == 0) && (a.chunk % EPQ == 0);
    if (vec && a.chunk % G == 0 && first_start + 32 * a.chunk <= in.length) {
        // all 32 rows whole (every item of an instance but its last): full tiles,
        // 32-byte stores at fixed strides, no per-row tests
        const int q = lane & 3, rsub = lane >> 2;
        T *dst0 = out + row0 + (uint64_t)q * EPQ;  // row r at dst0 + r chunk
        for (uint64_t done = 0; done < a.chunk; done += G) {
#pragma unroll
            for (int j = 0; j < G; j += VPL) {
                if constexpr (sizeof(T) == 4) {
                    T x[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) x[e] = bconvert<SRNG_MRG32K3A, OUT>(srng::mrg::step(s0, s1, s2, s3, s4, s5));
                    *reinterpret_cast<uint4 *>(&my[j]) = *reinterpret_cast<uint4 *>(x);
                } else {
                    double2 v;
                    v.x = bconvert<SRNG_MRG32K3A, OUT>(srng::mrg::step(s0, s1, s2, s3, s4, s5));
                    v.y = bconvert<SRNG_MRG32K3A, OUT>(srng::mrg::step(s0, s1, s2, s3, s4, s5));
                    *reinterpret_cast<double2 *>(&my[j]) = v;
                }
            }
            __syncwarp();
#pragma unroll
            for (int r0 = 0; r0 < 32; r0 += 8) {
                const int r = r0 + rsub;
                const T *src = &sm.tile[warp][r * RS + q * EPQ];
                bst256(dst0 + (uint64_t)r * a.chunk + done, *reinterpret_cast<const uint4 *>(src),
                       *reinterpret_cast<const uint4 *>(src + VPL));
            }
            __syncwarp();
        }
        return;
    }
    const uint32_t max_tiles = (uint32_t)((min(a.chunk, in.length - first_start) + G - 1) / G);  // row 0 is the longest
    for (uint32_t g = 0; g < max_tiles; ++g) {
        const uint64_t done = (uint64_t)g * G;
        const uint32_t rl = len > done ? (uint32_t)min((uint64_t)G, len - done) : 0u;
        auto fill = [&](uint32_t j) {  // VPL values of this lane's row into the tile
            if constexpr (sizeof(T) == 4) {
                T x[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) x[e] = bconvert<SRNG_MRG32K3A, OUT>(srng::mrg::step(s0, s1, s2, s3, s4, s5));
                *reinterpret_cast<uint4 *>(&my[j]) = *reinterpret_cast<uint4 *>(x);
            } else {
                double2 v;
                v.x = bconvert<SRNG_MRG32K3A, OUT>(srng::mrg::step(s0, s1, s2, s3, s4, s5));
                v.y = bconvert<SRNG_MRG32K3A, OUT>(srng::mrg::step(s0, s1, s2, s3, s4, s5));
                *reinterpret_cast<double2 *>(&my[j]) = v;
            }
        };
        if (rl == (uint32_t)G) {  // a full tile row: unrolled, so steps and stores interleave
#pragma unroll
            for (int j = 0; j < G; j += VPL) fill((uint32_t)j);
        } else {
            for (uint32_t j = 0; j < rl; j += VPL) fill(j);
        }
        __syncwarp();
        if (vec) {
            const int q = lane & 3, rsub = lane >> 2;
#pragma unroll
            for (int r0 = 0; r0 < 32; r0 += 8) {
                const int r = r0 + rsub;
                const uint64_t rstart = first_start + (uint64_t)r * a.chunk;  // draw index of the row
                if (rstart >= in.length) continue;
                const uint64_t rlen = min(a.chunk, in.length - rstart);
                const uint64_t e = done + (uint64_t)q * EPQ;                  // element within the row
                if (e >= rlen) continue;
                const T *src = &sm.tile[warp][r * RS + q * EPQ];
                T *dst = out + row0 + (uint64_t)r * a.chunk + e;
                if (e + EPQ <= rlen) {
                    bst256(dst, *reinterpret_cast<const uint4 *>(src), *reinterpret_cast<const uint4 *>(src + VPL));
                } else {
                    for (uint64_t x = 0; x < rlen - e; ++x) dst[x] = src[x];
                }
            }
        } else {
            constexpr int LPR = G, RPI = 32 / LPR;
            const int qe = lane % LPR, rsub = lane / LPR;
            for (int r0 = 0; r0 < 32; r0 += RPI) {
                const int r = r0 + rsub;
                const uint64_t rstart = first_start + (uint64_t)r * a.chunk;
                if (rstart >= in.length) continue;
                const uint64_t rlen = min(a.chunk, in.length - rstart);
                const uint64_t e = done + qe;
                if (e < rlen) out[row0 + (uint64_t)r * a.chunk + e] = sm.tile[warp][r * RS + qe];
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------- Philox work item
// Block q of an instance's stream (x0, x1 = q on entry), and the block pair
// (q, q + 1), for the instance's cipher (uniform over the warp).
__device__ __forceinline__ void item_block(int cipher, uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3,
                                           uint32_t kk0, uint32_t kk1, uint32_t c2, uint32_t c3)
{
    if (cipher == kCipherThreefry) cb_block<kCipherThreefry>(x0, x1, x2, x3, kk0, kk1, c2, c3);
    else if (cipher == kCipherThreefry64) cb_block<kCipherThreefry64>(x0, x1, x2, x3, kk0, kk1, c2, c3);
    else cb_block<kCipherPhilox>(x0, x1, x2, x3, kk0, kk1, c2, c3);
}
__device__ __forceinline__ void item_pair(int cipher, uint64_t q, uint32_t *w, uint32_t kk0, uint32_t kk1, uint32_t c2,
                                          uint32_t c3)
{
    if (cipher == kCipherThreefry) cb_pair<kCipherThreefry>(q, w, kk0, kk1, c2, c3);
    else if (cipher == kCipherThreefry64) cb_pair<kCipherThreefry64>(q, w, kk0, kk1, c2, c3);
    else cb_pair<kCipherPhilox>(q, w, kk0, kk1, c2, c3);
}

// Lane l computes pairs of adjacent blocks; eight values per pair go out as
// 32-byte stores when inside the instance and aligned, else element stores.
template <int OUT, bool PHILOX_ONLY = false>
__device__ void philox_item(const BatchArgs &a, uint32_t ii, uint32_t seg, int lane)
{
    using T = typename OutType<OUT>::T;
    const BatchInst &in = a.inst[ii];
    const uint64_t p0 = in.pos;
    const uint32_t al = (uint32_t)p0 & 3u;
    const uint64_t q0 = p0 >> 2;
    const uint64_t nb = (al + in.length + 3) >> 2;
    const uint64_t b0 = (uint64_t)seg * 32 * a.lane_blocks;
    const uint32_t c2 = (uint32_t)in.ctr_hi, c3 = (uint32_t)(in.ctr_hi >> 32);
    const int tf = PHILOX_ONLY ? kCipherPhilox  // a kernel for Philox items alone holds no Threefry code
                 : in.gen == SRNG_THREEFRY4X32_20 ? kCipherThreefry
                 : in.gen == SRNG_THREEFRY4X64_20 ? kCipherThreefry64 : kCipherPhilox;  // uniform over the warp
    const uint64_t L = in.length;
    if (a.mode == SRNG_BATCH_FUSED_PI) {
        uint32_t hits = 0;
        // the four words of 4-word group b (draw index of word 0: k0) and the
        // next group's word 0 when the pairs straddle (odd start)
        auto count_group = [&](uint64_t b, const uint32_t *x, auto next_word0) {
            const int64_t k0 = (int64_t)(b * 4) - al;
            if ((al & 1) == 0) {
                // pairs are (word 0, word 1) and (word 2, word 3)
                if (k0 >= 0 && (uint64_t)k0 + 1 < L) hits += hit_philox(x[0], x[1]);
                if (k0 + 2 >= 0 && (uint64_t)(k0 + 2) + 1 < L) hits += hit_philox(x[2], x[3]);
            } else {
                // odd start: pairs (word 1, word 2) and (word 3, next group's word 0)
                if (k0 + 1 >= 0 && (uint64_t)(k0 + 1) + 1 < L) hits += hit_philox(x[1], x[2]);
                if (k0 + 3 >= 0 && (uint64_t)(k0 + 3) + 1 < L) hits += hit_philox(x[3], next_word0());
            }
        };
        if (tf == kCipherThreefry64) {
            // One Threefry4x64 block holds the 4-word groups 2Q and 2Q + 1: each
            // lane takes whole blocks and counts the halves inside this item's
            // groups [b0, b_end), so a block is computed once (once more for the
            // straddling pair of an odd start at its upper half).
            const uint64_t b_end = min(b0 + (uint64_t)32 * a.lane_blocks, nb);
            const uint64_t kk = (uint64_t)in.key1 << 32 | in.key0, sd = (uint64_t)c3 << 32 | c2;
            for (uint64_t Q = ((q0 + b0) >> 1) + lane; 2 * Q < q0 + b_end; Q += 32) {
                uint32_t w[8];
                srng::threefry64::words(Q, kk, sd, w);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint64_t g = 2 * Q + h;  // absolute group
                    if (g < q0 + b0 || g - q0 >= b_end) continue;
                    count_group(g - q0, w + 4 * h, [&]() {
                        if (h == 0) return w[4];
                        uint32_t v[8];
                        srng::threefry64::words(Q + 1, kk, sd, v);
                        return v[0];
                    });
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) hits += __shfl_down_sync(0xffffffffu, hits, o);
            if (lane == 0 && hits) atomicAdd(reinterpret_cast<unsigned long long *>(a.out) + ii, (unsigned long long)hits);
            return;
        }
        for (uint32_t u = 0; u < a.lane_blocks; ++u) {
            const uint64_t b = b0 + (uint64_t)u * 32 + lane;
            if (b >= nb) break;
            const uint64_t q = q0 + b;
            uint32_t x[4] = {(uint32_t)q, (uint32_t)(q >> 32), 0u, 0u};
            item_block(tf, x[0], x[1], x[2], x[3], in.key0, in.key1, c2, c3);
            count_group(b, x, [&]() {
                const uint64_t qn = q + 1;
                uint32_t y0 = (uint32_t)qn, y1 = (uint32_t)(qn >> 32), y2, y3;
                item_block(tf, y0, y1, y2, y3, in.key0, in.key1, c2, c3);
                return y0;
            });
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hits += __shfl_down_sync(0xffffffffu, hits, o);
        if (lane == 0 && hits) atomicAdd(reinterpret_cast<unsigned long long *>(a.out) + ii, (unsigned long long)hits);
        return;
    }
    T *row = static_cast<T *>(a.out) + in.out_offset;
    // draws this item may write: its own blocks only (an odd lane_blocks leaves
    // the last pair half outside), and the instance's length
    const int64_t lim = min((int64_t)L, (int64_t)(4 * (b0 + 32ull * a.lane_blocks)) - (int64_t)al);
    auto store_pair = [&](uint64_t b, const uint32_t *w) {  // the eight values of blocks b, b + 1
        const int64_t k0 = (int64_t)(b * 4) - al;
        T v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = bconvert<SRNG_PHILOX4X32_10, OUT>(w[j]);
        if (k0 >= 0 && k0 + 8 <= lim && ((reinterpret_cast<uintptr_t>(row + k0) & 31) == 0)) {
            const uint4 *p = reinterpret_cast<const uint4 *>(v);
            bst256(row + k0, p[0], p[1]);
            if constexpr (sizeof(T) == 8) bst256(row + k0 + 4, p[2], p[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int64_t k = k0 + j;
                if (k >= 0 && k < lim) row[k] = v[j];
            }
        }
    };
    // PP pairs per lane in flight (2 PP independent blocks); pairs past the end
    // of the item are computed and then not stored
    constexpr int PP = 4;
    for (uint32_t u = 0; u < a.lane_blocks; u += 2 * PP) {
        const uint64_t b = b0 + (uint64_t)u * 32 + 2 * lane;  // this lane's pairs: b + 64 p, b + 64 p + 1
        if (b >= nb) break;
        uint32_t w[PP][8];
#pragma unroll
        for (int p = 0; p < PP; ++p) item_pair(tf, q0 + b + 64 * p, w[p], in.key0, in.key1, c2, c3);
#pragma unroll
        for (int p = 0; p < PP; ++p)
            if (u + 2 * p < a.lane_blocks && b + 64 * p < nb) store_pair(b + 64 * p, w[p]);
    }
}

// FAM: which work items the kernel holds code for -- MRG32k3a items or
// counter-based (Philox, Threefry) items.  A plan launches one kernel per family
// present: each carries half the code, so fewer instruction-cache misses, and
// its own register count and occupancy.
enum { kFamMrg = 1, kFamCounter = 2, kFamPhilox = 3 };

template <int OUT, int FAM>
__global__ void __launch_bounds__(kWarps * 32, FAM == kFamMrg ? (OUT == SRNG_OUT_F64 ? 2 : 4) : FAM == kFamPhilox ? 3 : 4)
    k_batch(const BatchArgs a, const __grid_constant__ JumpTable tab)
{
    __shared__ __align__(16) Smem<OUT> sm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(a.counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= a.n_items) break;
        const uint2 item = a.items[it];
        if constexpr (FAM == kFamMrg) mrg_item<OUT>(a, tab, it, item.x, item.y, sm, warp, lane);
        else philox_item<OUT, FAM == kFamPhilox>(a, item.x, item.y, lane);
    }
}

// Instance start states: MRG32k3a = A^offset applied to the stream's state
// (J_k = A^(2^k)); Philox = stream position + offset.  `zero`, if given, is a
// work counter set to 0 here (one stream operation less than a memset).
__global__ void __launch_bounds__(256)
    k_batch_setup(BatchInst *inst, uint64_t n, const __grid_constant__ JumpTable tab, uint32_t *zero)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && zero) *zero = 0u;
    if (i >= n) return;
    BatchInst &in = inst[i];
    if (in.gen == SRNG_MRG32K3A) {
        const uint64_t ns = in.src_ns, s = in.stream;
        uint32_t s0 = in.src_state[s], s1 = in.src_state[ns + s], s2 = in.src_state[2 * ns + s];
        uint32_t s3 = in.src_state[3 * ns + s], s4 = in.src_state[4 * ns + s], s5 = in.src_state[5 * ns + s];
        for (int k = 0; k < 64; ++k)
            if ((in.offset >> k) & 1) srng::mrg::jump(tab.m[k], s0, s1, s2, s3, s4, s5);
        in.st[0] = s0; in.st[1] = s1; in.st[2] = s2; in.st[3] = s3; in.st[4] = s4; in.st[5] = s5;
    } else {
        in.pos = in.src_pos[in.stream] + in.offset;
    }
}

// State at each MRG32k3a item's first chunk: the instance's start state moved
// by J_k = A^(chunk 2^k) for the set bits of the first chunk (a multiple of 32).
__global__ void __launch_bounds__(256)
    k_batch_item_states(const BatchInst *inst, const uint2 *items, uint64_t n, const __grid_constant__ JumpTable tab,
                        uint32_t *item_state)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint2 item = items[i];
    const BatchInst &in = inst[item.x];
    uint32_t s0 = in.st[0], s1 = in.st[1], s2 = in.st[2], s3 = in.st[3], s4 = in.st[4], s5 = in.st[5];
    for (int k = 0; k < 32; ++k)
        if ((item.y >> k) & 1) srng::mrg::jump(tab.m[k], s0, s1, s2, s3, s4, s5);
    uint32_t *o = item_state + 6 * i;
    o[0] = s0; o[1] = s1; o[2] = s2; o[3] = s3; o[4] = s4; o[5] = s5;
}

// The same state straight from the stream's state, for small steps of the
// server: A^offset (J_k = A^(2^k), `unit`) then A^(chunk first) (`tab`) per
// item, so no set-up kernel runs before it (each item repeats its instance's
// offset jump); `zero` is the step's work counter, set to 0 here.
__global__ void __launch_bounds__(256)
    k_batch_item_states_direct(const BatchInst *inst, const uint2 *items, uint64_t n,
                               const __grid_constant__ JumpTable unit, const __grid_constant__ JumpTable tab,
                               uint32_t *item_state, uint32_t *zero)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && zero) *zero = 0u;
    if (i >= n) return;
    const uint2 item = items[i];
    const BatchInst &in = inst[item.x];
    const uint64_t ns = in.src_ns, s = in.stream;
    uint32_t s0 = in.src_state[s], s1 = in.src_state[ns + s], s2 = in.src_state[2 * ns + s];
    uint32_t s3 = in.src_state[3 * ns + s], s4 = in.src_state[4 * ns + s], s5 = in.src_state[5 * ns + s];
    for (int k = 0; k < 64; ++k)
        if ((in.offset >> k) & 1) srng::mrg::jump(unit.m[k], s0, s1, s2, s3, s4, s5);
    for (int k = 0; k < 32; ++k)
        if ((item.y >> k) & 1) srng::mrg::jump(tab.m[k], s0, s1, s2, s3, s4, s5);
    uint32_t *o = item_state + 6 * i;
    o[0] = s0; o[1] = s1; o[2] = s2; o[3] = s3; o[4] = s4; o[5] = s5;
}

// J_k = A^(2^k), k < 64 (built once).
const JumpTable &unit_jump_table()
{
    static std::once_flag once;
    static JumpTable unit_tab;
    std::call_once(once, [] {
        for (int k = 0; k < 64; ++k) memcpy(unit_tab.m[k], mat_pow2(k).a, sizeof unit_tab.m[k]);
    });
    return unit_tab;
}

}  // namespace

// Host-side plan.
struct BatchPlanImpl {
    int device;
    srng_batch_mode mode;
    srng_out type;
    uint64_t n_inst, n_items;
    BatchInst *d_inst = nullptr;
    uint2 *d_items = nullptr;
    uint32_t *d_item_state = nullptr;        // MRG32k3a items' first-chunk states
    uint32_t *d_lane_tab = nullptr;          // A^(chunk l), l < 32
    uint32_t *d_counter = nullptr;           // one per family kernel
    void *out = nullptr;
    BatchArgs args[2];                       // [0] MRG32k3a items, [1] counter-based items
    JumpTable chunk_tab;
    unsigned grid[2] = {0, 0};
    int cfam = 2;                            // kernel family of the counter-based items (kFamCounter / kFamPhilox)
    cudaStream_t side = nullptr;             // capture fork for the second kernel
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t kernels() const { return (args[0].n_items ? 1u : 0u) + (args[1].n_items ? 1u : 0u); }
};

}  // namespace srng_impl

struct srng_batch_plan {
    srng_impl::BatchPlanImpl p;
};

using namespace srng_impl;

namespace srng_impl {

static void plan_free(srng_batch_plan *pl)
{
    if (!pl) return;
    BatchPlanImpl &p = pl->p;
    if (p.exec) cudaGraphExecDestroy(p.exec);
    if (p.graph) cudaGraphDestroy(p.graph);
    if (p.d_inst) cudaFree(p.d_inst);
    if (p.d_items) cudaFree(p.d_items);
    if (p.d_item_state) cudaFree(p.d_item_state);
    if (p.d_lane_tab) cudaFree(p.d_lane_tab);
    if (p.d_counter) cudaFree(p.d_counter);
    if (p.side) cudaStreamDestroy(p.side);
    if (p.fork) cudaEventDestroy(p.fork);
    if (p.join) cudaEventDestroy(p.join);
    delete pl;
}

template <int FAM>
static void launch_fam(srng_out type, unsigned grid, const BatchArgs &a, const JumpTable &tab, cudaStream_t s)
{
    switch (type) {
    case SRNG_OUT_U32: k_batch<SRNG_OUT_U32, FAM><<<grid, kWarps * 32, 0, s>>>(a, tab); break;
    case SRNG_OUT_F32: k_batch<SRNG_OUT_F32, FAM><<<grid, kWarps * 32, 0, s>>>(a, tab); break;
    default: k_batch<SRNG_OUT_F64, FAM><<<grid, kWarps * 32, 0, s>>>(a, tab); break;
    }
}

// {reset counters, zero counts} then the family kernels; with both families the
// counter-based kernel goes on a forked stream so the two are independent graph
// nodes (its blocks take SMs as the MRG32k3a kernel's blocks finish).
static cudaError_t enqueue_batch(const BatchPlanImpl &p, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(p.d_counter, 0, 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if (p.mode == SRNG_BATCH_FUSED_PI && p.n_inst) {
        e = cudaMemsetAsync(p.out, 0, p.n_inst * sizeof(int64_t), s);
        if (e != cudaSuccess) return e;
    }
    const bool m = p.args[0].n_items > 0, c = p.args[1].n_items > 0;
    if (m && c) {
        if ((e = cudaEventRecord(p.fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(p.side, p.fork, 0)) != cudaSuccess) return e;
        launch_fam<kFamMrg>(p.type, p.grid[0], p.args[0], p.chunk_tab, s);
        if (p.cfam == kFamPhilox) launch_fam<kFamPhilox>(p.type, p.grid[1], p.args[1], p.chunk_tab, p.side);
        else launch_fam<kFamCounter>(p.type, p.grid[1], p.args[1], p.chunk_tab, p.side);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(p.join, p.side)) != cudaSuccess) return e;
        return cudaStreamWaitEvent(s, p.join, 0);
    }
    if (m) launch_fam<kFamMrg>(p.type, p.grid[0], p.args[0], p.chunk_tab, s);
    if (c) {
        if (p.cfam == kFamPhilox) launch_fam<kFamPhilox>(p.type, p.grid[1], p.args[1], p.chunk_tab, s);
        else launch_fam<kFamCounter>(p.type, p.grid[1], p.args[1], p.chunk_tab, s);
    }
    return cudaGetLastError();
}

template <int FAM>
static int occupancy_blocks_fam(srng_out type)
{
    int nb = 0;
    switch (type) {
    case SRNG_OUT_U32: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<SRNG_OUT_U32, FAM>, kWarps * 32, 0); break;
    case SRNG_OUT_F32: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<SRNG_OUT_F32, FAM>, kWarps * 32, 0); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<SRNG_OUT_F64, FAM>, kWarps * 32, 0); break;
    }
    return nb > 0 ? nb : 1;
}


cudaError_t launch_batch_setup(BatchInst *d_inst, uint64_t n, cudaStream_t s, uint32_t *zero)
{
    if (n == 0) return cudaSuccess;
    k_batch_setup<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_inst, n, unit_jump_table(), zero);
    return cudaGetLastError();
}

cudaError_t launch_batch_item_states_direct(const BatchInst *d_inst, const uint2 *d_items, uint64_t n,
                                            const JumpTable &chunk_tab, uint32_t *item_state, uint32_t *zero,
                                            cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_batch_item_states_direct<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_inst, d_items, n, unit_jump_table(),
                                                                          chunk_tab, item_state, zero);
    return cudaGetLastError();
}

cudaError_t launch_batch_item_states(const BatchInst *d_inst, const uint2 *d_items, uint64_t n,
                                     const JumpTable &chunk_tab, uint32_t *item_state, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_batch_item_states<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_inst, d_items, n, chunk_tab, item_state);
    return cudaGetLastError();
}

void lane_jump_table(uint64_t chunk, uint32_t out[32 * 18])
{
    const MatPair c = mat_pow_shifted(0, chunk, 0);
    MatPair m = mat_identity();
    for (int l = 0; l < 32; ++l) {
        memcpy(out + 18 * l, m.a, sizeof m.a);
        m = mat_mul(m, c);
    }
}

cudaError_t launch_batch(const BatchArgs &a, srng_out type, BatchFamily fam, const JumpTable &chunk_tab, unsigned grid,
                         cudaStream_t s)
{
    if (a.n_items == 0) return cudaSuccess;
    if (fam == kBatchMrg) launch_fam<kFamMrg>(type, grid, a, chunk_tab, s);
    else if (fam == kBatchPhilox) launch_fam<kFamPhilox>(type, grid, a, chunk_tab, s);
    else launch_fam<kFamCounter>(type, grid, a, chunk_tab, s);
    return cudaGetLastError();
}

int batch_blocks_per_sm(srng_out type, BatchFamily fam)
{
    return fam == kBatchMrg ? occupancy_blocks_fam<kFamMrg>(type)
         : fam == kBatchPhilox ? occupancy_blocks_fam<kFamPhilox>(type) : occupancy_blocks_fam<kFamCounter>(type);
}

void chunk_jump_table(uint64_t chunk, JumpTable *out)
{
    MatPair m = mat_pow_shifted(0, chunk, 0);
    for (int k = 0; k < 64; ++k) {
        memcpy(out->m[k], m.a, sizeof m.a);
        m = mat_mul(m, m);
    }
}

// Validate, build instance descriptors and the item list on the host.
srng_status batch_build(srng_set *const *sets, uint32_t n_sets, const srng_instance *inst, uint64_t n_inst,
                        srng_batch_mode mode, srng_out type, void *out_dev, const srng_tune &t,
                        std::vector<BatchInst> &hin, std::vector<uint2> &items, uint64_t &chunk,
                        uint64_t *n_mrg_items)
{
    std::vector<uint2> cb_items;  // counter-based items, placed after the MRG32k3a ones
    if (mode != SRNG_BATCH_WRITE && mode != SRNG_BATCH_FUSED_PI) return fail(SRNG_ERR_ARG, "unknown batch mode");
    if (type != SRNG_OUT_U32 && type != SRNG_OUT_F32 && type != SRNG_OUT_F64)
        return fail(SRNG_ERR_ARG, "unknown output type");
    if (n_inst && (!inst || !sets || n_sets == 0)) return fail(SRNG_ERR_ARG, "NULL instances or sets");
    if (n_inst >= (1ull << 32)) return fail(SRNG_ERR_ARG, "at most 2^32 - 1 instances");
    if (n_inst && !out_dev) return fail(SRNG_ERR_ARG, "output pointer is NULL");
    const size_t esz = type == SRNG_OUT_F64 ? 8 : 4;
    if (mode == SRNG_BATCH_WRITE && reinterpret_cast<uintptr_t>(out_dev) % esz)
        return fail(SRNG_ERR_ARG, "output pointer not aligned to the element size");
    if (mode == SRNG_BATCH_FUSED_PI && reinterpret_cast<uintptr_t>(out_dev) % 8)
        return fail(SRNG_ERR_ARG, "counts pointer not 8-byte aligned");
    chunk = t.chunk ? t.chunk : 512;
    const uint64_t lane_blocks = t.lane_blocks ? t.lane_blocks : 64;
    hin.resize(n_inst);
    for (uint64_t i = 0; i < n_inst; ++i) {
        const srng_instance &x = inst[i];
        if (x.set_index >= n_sets || !sets[x.set_index])
            return fail(SRNG_ERR_ARG, "instance " + std::to_string(i) + ": bad set index");
        const srng_set *s = sets[x.set_index];
        if (s->gen == SRNG_TINYMT32) return fail(SRNG_ERR_UNSUPPORTED, "TinyMT32 sets are not batched");
        if (x.stream >= s->n_streams) return fail(SRNG_ERR_RANGE, "instance " + std::to_string(i) + ": stream outside its set");
        if (x.length > (1ull << 48)) return fail(SRNG_ERR_ARG, "instance " + std::to_string(i) + ": length above 2^48");
        if (s->gen == SRNG_PHILOX4X32_10 && (x.offset > UINT64_MAX - s->max_pos ||
                                             x.length > UINT64_MAX - s->max_pos - x.offset))
            return fail(SRNG_ERR_RANGE, "instance " + std::to_string(i) + ": Philox position would pass 2^64 - 1");
        BatchInst b;
        memset(&b, 0, sizeof b);
        b.gen = inst_gen(s);
        const uint64_t gs = s->stream_base + x.stream;  // stream number
        b.key0 = s->keyed ? (uint32_t)gs : s->key0;
        b.key1 = s->keyed ? (uint32_t)(gs >> 32) : s->key1;
        b.ctr_hi = s->keyed ? ((uint64_t)s->key1 << 32 | s->key0) : gs;
        b.stream = x.stream;
        b.offset = x.offset;
        b.length = x.length;
        b.out_offset = x.out_offset;
        b.src_state = s->d_state;
        b.src_ns = s->n_streams;
        b.src_pos = s->d_pos;
        hin[i] = b;
        if (x.length == 0) continue;
        if (s->gen == SRNG_MRG32K3A) {
            const uint64_t nch = (x.length + chunk - 1) / chunk;
            if (nch > (1ull << 32)) return fail(SRNG_ERR_ARG, "instance too long for the chunk size");
            for (uint64_t c = 0; c < nch; c += 32) items.push_back(make_uint2((uint32_t)i, (uint32_t)c));
        } else {
            const uint64_t nb = (x.length + 3) / 4 + 1;
            const uint64_t per = 32 * lane_blocks;
            const uint64_t nseg = (nb + per - 1) / per;
            if (nseg > (1ull << 32)) return fail(SRNG_ERR_ARG, "instance too long");
            for (uint64_t g = 0; g < nseg; ++g) cb_items.push_back(make_uint2((uint32_t)i, (uint32_t)g));
        }
    }
    if (n_mrg_items) *n_mrg_items = items.size();
    items.insert(items.end(), cb_items.begin(), cb_items.end());
    if (items.size() >= (1ull << 32)) return fail(SRNG_ERR_ARG, "too many work items");
    return SRNG_OK;
}

}  // namespace srng_impl

extern "C" {

srng_status srng_batch_plan_create(srng_batch_plan **out, srng_set *const *sets, uint32_t n_sets,
                                   const srng_instance *inst, uint64_t n_inst, srng_batch_mode mode, srng_out type,
                                   void *out_dev, const srng_tune *tune, void *cuda_stream)
{
    clear_error();
    if (!out) return fail(SRNG_ERR_ARG, "out is NULL");
    *out = nullptr;
    srng_status st = check_tune(tune);
    if (st) return st;
    DeviceInfo dev;
    if ((st = current_device(&dev))) return st;
    const srng_tune t = effective_tune(SRNG_MRG32K3A, type == SRNG_OUT_F64 ? SRNG_OUT_F64 : type, tune);
    std::vector<BatchInst> hin;
    std::vector<uint2> items;
    uint64_t chunk = 0, n_mrg = 0;
    if ((st = batch_build(sets, n_sets, inst, n_inst, mode, type, out_dev, t, hin, items, chunk, &n_mrg))) return st;

    srng_batch_plan *pl = new (std::nothrow) srng_batch_plan();
    if (!pl) return fail(SRNG_ERR_OOM, "host allocation failed");
    BatchPlanImpl &p = pl->p;
    p.device = dev.device;
    p.mode = mode;
    p.type = type;
    p.n_inst = n_inst;
    p.n_items = items.size();
    p.out = out_dev;
    p.cfam = kFamPhilox;  // a kernel with Philox code alone, unless a Threefry instance is present
    for (const BatchInst &b : hin)
        if (b.length && (b.gen == SRNG_THREEFRY4X32_20 || b.gen == SRNG_THREEFRY4X64_20)) p.cfam = kFamCounter;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    cudaStream_t cap = nullptr;
    cudaError_t e;
#define PLAN_TRY(expr)                                                   \
    do {                                                                 \
        e = (expr);                                                      \
        if (e != cudaSuccess) { st = cuda_fail(e, #expr); goto bad; }    \
    } while (0)
    PLAN_TRY(cudaMalloc(&p.d_counter, 2 * sizeof(uint32_t)));
    PLAN_TRY(cudaStreamCreateWithFlags(&p.side, cudaStreamNonBlocking));
    PLAN_TRY(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming));
    PLAN_TRY(cudaEventCreateWithFlags(&p.join, cudaEventDisableTiming));
    if (n_inst) {
        PLAN_TRY(cudaMalloc(&p.d_inst, n_inst * sizeof(BatchInst)));
        PLAN_TRY(cudaMemcpyAsync(p.d_inst, hin.data(), n_inst * sizeof(BatchInst), cudaMemcpyHostToDevice, stream));
        {
            JumpTable unit_tab;  // J_k = A^(2^k)
            for (int k = 0; k < 64; ++k) memcpy(unit_tab.m[k], mat_pow2(k).a, sizeof unit_tab.m[k]);
            const unsigned g = (unsigned)((n_inst + 255) / 256);
            k_batch_setup<<<g, 256, 0, stream>>>(p.d_inst, n_inst, unit_tab, nullptr);
            PLAN_TRY(cudaGetLastError());
        }
    }
    if (p.n_items) {
        PLAN_TRY(cudaMalloc(&p.d_items, p.n_items * sizeof(uint2)));
        PLAN_TRY(cudaMemcpyAsync(p.d_items, items.data(), p.n_items * sizeof(uint2), cudaMemcpyHostToDevice, stream));
    }
    {
        MatPair m = mat_pow_shifted(0, chunk, 0);  // J_k = A^(chunk 2^k)
        for (int k = 0; k < 64; ++k) {
            memcpy(p.chunk_tab.m[k], m.a, sizeof m.a);
            m = mat_mul(m, m);
        }
    }
    if (n_mrg) {  // each MRG32k3a item's first-chunk state, and the lane table
        uint32_t lane_tab[32 * 18];
        lane_jump_table(chunk, lane_tab);
        PLAN_TRY(cudaMalloc(&p.d_lane_tab, sizeof lane_tab));
        PLAN_TRY(cudaMemcpyAsync(p.d_lane_tab, lane_tab, sizeof lane_tab, cudaMemcpyHostToDevice, stream));
        PLAN_TRY(cudaMalloc(&p.d_item_state, n_mrg * 6 * sizeof(uint32_t)));
        PLAN_TRY(launch_batch_item_states(p.d_inst, p.d_items, n_mrg, p.chunk_tab, p.d_item_state, stream));
    }
    for (int f = 0; f < 2; ++f) {  // [0] MRG32k3a items, [1] counter-based items
        BatchArgs &a = p.args[f];
        a.inst = p.d_inst;
        a.items = p.d_items ? p.d_items + (f ? n_mrg : 0) : nullptr;
        a.counter = p.d_counter + f;
        a.n_items = f ? p.n_items - n_mrg : n_mrg;
        a.chunk = chunk;
        a.lane_blocks = t.lane_blocks ? t.lane_blocks : 64;
        a.mode = mode;
        a.out = out_dev;
        a.item_state = f ? nullptr : p.d_item_state;
        a.lane_tab = f ? nullptr : p.d_lane_tab;
        int per_sm = !f ? occupancy_blocks_fam<kFamMrg>(type)
                   : p.cfam == kFamPhilox ? occupancy_blocks_fam<kFamPhilox>(type) : occupancy_blocks_fam<kFamCounter>(type);
        if (tune && tune->blocks_per_sm) per_sm = std::min<int>(per_sm, (int)tune->blocks_per_sm);
        const uint64_t want = (a.n_items + kWarps - 1) / kWarps;
        uint64_t g = (uint64_t)dev.sm_count * per_sm;
        if (g > want) g = want;
        p.grid[f] = (unsigned)std::max<uint64_t>(1, g);
    }
    PLAN_TRY(cudaStreamSynchronize(stream));
    // Capture {reset counter, zero counts, persistent kernel} once.
    PLAN_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    PLAN_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    e = enqueue_batch(p, cap);
    {
        cudaError_t e2 = cudaStreamEndCapture(cap, &p.graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) { st = cuda_fail(e, "graph capture of the batch launch"); goto bad; }
    PLAN_TRY(cudaGraphInstantiate(&p.exec, p.graph, 0));
    cudaStreamDestroy(cap);
    *out = pl;
    return SRNG_OK;
bad:
    if (cap) cudaStreamDestroy(cap);
    plan_free(pl);
    return st;
#undef PLAN_TRY
}

srng_status srng_batch_plan_launch(srng_batch_plan *plan, void *cuda_stream)
{
    clear_error();
    if (!plan) return fail(SRNG_ERR_ARG, "plan is NULL");
    SRNG_CUDA_TRY(cudaGraphLaunch(plan->p.exec, static_cast<cudaStream_t>(cuda_stream)));
    return SRNG_OK;
}

srng_status srng_batch_plan_info(const srng_batch_plan *plan, uint64_t *n_work_items, uint32_t *kernels_per_launch)
{
    clear_error();
    if (!plan) return fail(SRNG_ERR_ARG, "plan is NULL");
    if (n_work_items) *n_work_items = plan->p.n_items;
    if (kernels_per_launch) *kernels_per_launch = plan->p.kernels();
    return SRNG_OK;
}

srng_status srng_batch_plan_destroy(srng_batch_plan *plan)
{
    clear_error();
    if (!plan) return SRNG_OK;
    cudaDeviceSynchronize();
    plan_free(plan);
    return SRNG_OK;
}

srng_status srng_batch_run(srng_set *const *sets, uint32_t n_sets, const srng_instance *inst, uint64_t n_inst,
                           srng_batch_mode mode, srng_out type, void *out_dev, void *cuda_stream)
{
    srng_batch_plan *plan = nullptr;
    srng_status st = srng_batch_plan_create(&plan, sets, n_sets, inst, n_inst, mode, type, out_dev, nullptr, cuda_stream);
    if (st) return st;
    st = srng_batch_plan_launch(plan, cuda_stream);
    if (st == SRNG_OK) {
        cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize(batch)");
    }
    srng_batch_plan_destroy(plan);
    return st;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// srng_batch_run_static: the batched launch without any allocation.
//
// The paper has no counterpart to this entry point.  It exists for callers
// that must not allocate device memory per call: code whose device memory is
// owned by another allocator (a framework's caching allocator or a plugin
// host that forbids cudaMalloc), and latency-critical loops that cannot pay
// for cudaMalloc / cudaFree and the device synchronisation cudaFree implies.
// Its scratch (instance descriptors, per-instance work-item prefix sums, the
// work counter) lives in one file-scope __device__ array of fixed size, which
// every GPU that loads this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace srng_impl {

namespace {

constexpr uint32_t kStaticMaxInst = SRNG_BATCH_STATIC_MAX_INSTANCES;
constexpr uint32_t kStaticMaxSets = SRNG_BATCH_STATIC_MAX_SETS;
constexpr uint64_t kStaticChunk = 512;       // MRG32k3a draws per lane-chunk
constexpr uint32_t kStaticLaneBlocks = 64;   // Philox blocks per lane per work item
// Work items of one call: the work counter, the total and the item numbers are
// 32-bit, and every warp adds one to the counter past the total before it
// stops, so the total stays far below 2^32.
constexpr uint64_t kStaticMaxItems = 1ull << 31;

constexpr size_t round256(size_t x) { return (x + 255) / 256 * 256; }
// Layout: [0,4) work counter, [4,8) total work items, then the prefix sums of
// work items per instance (kStaticMaxInst + 1 words), the caller's instances
// as copied, and the device-side instance descriptors.
constexpr size_t kOffPrefix = 256;
constexpr size_t kOffRaw = round256(kOffPrefix + 8 * (size_t)(kStaticMaxInst + 1));
constexpr size_t kOffInst = round256(kOffRaw + sizeof(srng_instance) * (size_t)kStaticMaxInst);
constexpr size_t kStaticBytes = round256(kOffInst + sizeof(BatchInst) * (size_t)kStaticMaxInst);

static __device__ __align__(256) unsigned char g_batch_scratch[kStaticBytes];

struct StaticSets {
    uint32_t gen[kStaticMaxSets];
    uint32_t key0[kStaticMaxSets], key1[kStaticMaxSets];
    uint32_t keyed[kStaticMaxSets];
    uint64_t base[kStaticMaxSets];
    const uint32_t *state[kStaticMaxSets];
    uint64_t ns[kStaticMaxSets];
    const uint64_t *pos[kStaticMaxSets];
};

// One thread per instance: descriptor (start state by jump-ahead, as in
// k_batch_setup) and its number of work items.
__global__ void __launch_bounds__(256)
    k_static_setup(unsigned char *scr, uint32_t n_inst, const StaticSets sets, const __grid_constant__ JumpTable unit)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    const srng_instance r = reinterpret_cast<const srng_instance *>(scr + kOffRaw)[i];
    const uint32_t si = r.set_index;
    BatchInst b;
    memset(&b, 0, sizeof b);
    b.gen = sets.gen[si];
    const uint64_t gs = sets.base[si] + r.stream;  // stream number
    b.key0 = sets.keyed[si] ? (uint32_t)gs : sets.key0[si];
    b.key1 = sets.keyed[si] ? (uint32_t)(gs >> 32) : sets.key1[si];
    b.ctr_hi = sets.keyed[si] ? ((uint64_t)sets.key1[si] << 32 | sets.key0[si]) : gs;
    b.stream = r.stream;
    b.offset = r.offset;
    b.length = r.length;
    b.out_offset = r.out_offset;
    uint64_t items = 0;
    if (b.gen == SRNG_MRG32K3A) {
        const uint32_t *st = sets.state[si];
        const uint64_t ns = sets.ns[si], s = r.stream;
        uint32_t s0 = st[s], s1 = st[ns + s], s2 = st[2 * ns + s], s3 = st[3 * ns + s], s4 = st[4 * ns + s],
                 s5 = st[5 * ns + s];
        for (int k = 0; k < 64; ++k)
            if ((r.offset >> k) & 1) srng::mrg::jump(unit.m[k], s0, s1, s2, s3, s4, s5);
        b.st[0] = s0; b.st[1] = s1; b.st[2] = s2; b.st[3] = s3; b.st[4] = s4; b.st[5] = s5;
        const uint64_t nch = (r.length + kStaticChunk - 1) / kStaticChunk;
        items = (nch + 31) / 32;
    } else {
        b.pos = sets.pos[si][r.stream] + r.offset;
        if (r.length) {
            const uint64_t nb = (r.length + 3) / 4 + 1, per = 32ull * kStaticLaneBlocks;
            items = (nb + per - 1) / per;
        }
    }
    reinterpret_cast<BatchInst *>(scr + kOffInst)[i] = b;
    reinterpret_cast<uint64_t *>(scr + kOffPrefix)[i + 1] = items;
}

// One block: exclusive prefix sums of the work items, the total, and the
// zeroing of what must start at zero (work counter; hit counts in FUSED_PI).
__global__ void __launch_bounds__(1024) k_static_scan(unsigned char *scr, uint32_t n_inst, int64_t *counts)
{
    __shared__ uint64_t warp_sums[32];
    uint64_t *prefix = reinterpret_cast<uint64_t *>(scr + kOffPrefix);
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr uint32_t kPer = (kStaticMaxInst + 1023) / 1024;  // consecutive elements per thread
    uint64_t v[kPer];
    uint64_t local = 0;
#pragma unroll
    for (uint32_t e = 0; e < kPer; ++e) {
        const uint32_t i = tid * kPer + e;
        v[e] = i < n_inst ? prefix[i + 1] : 0;
        local += v[e];
    }
    uint64_t incl = local;  // inclusive scan of the per-thread totals
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= (uint32_t)o) w += y;
        }
        warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    uint64_t run = incl - local + (warp ? warp_sums[warp - 1] : 0);  // exclusive start of this thread
#pragma unroll
    for (uint32_t e = 0; e < kPer; ++e) {
        const uint32_t i = tid * kPer + e;
        if (i < n_inst) prefix[i] = run;
        run += v[e];
    }
    if (tid == 1023) {
        prefix[n_inst] = run;  // total (run ends at the grand total on the last thread)
        reinterpret_cast<uint32_t *>(scr)[1] = (uint32_t)run;
        reinterpret_cast<uint32_t *>(scr)[0] = 0u;
    }
    if (counts)
        for (uint32_t i = tid; i < n_inst; i += 1024) counts[i] = 0;
}

template <int OUT>
__global__ void __launch_bounds__(kWarps * 32)
    k_batch_static(unsigned char *scr, uint32_t n_inst, BatchArgs a, const __grid_constant__ JumpTable tab)
{
    __shared__ __align__(16) Smem<OUT> sm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t *prefix = reinterpret_cast<const uint64_t *>(scr + kOffPrefix);
    const uint32_t total = reinterpret_cast<const volatile uint32_t *>(scr)[1];
    a.inst = reinterpret_cast<const BatchInst *>(scr + kOffInst);
    a.counter = reinterpret_cast<uint32_t *>(scr);
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(a.counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= total) break;
        uint32_t lo = 0, hi = n_inst;  // largest lo < n_inst with prefix[lo] <= it
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (prefix[mid] <= it) lo = mid;
            else hi = mid;
        }
        const uint32_t j = it - (uint32_t)prefix[lo];
        if (a.inst[lo].gen == SRNG_MRG32K3A) mrg_item<OUT>(a, tab, it, lo, 32u * j, sm, warp, lane);
        else philox_item<OUT>(a, lo, j, lane);
    }
}

// Per-device set-up: the scratch array's device address, the persistent grid
// size, and the two jump tables (computed once per process, on the stack of
// the set-up call, no heap use).
struct StaticDevice {
    bool ready;
    unsigned char *scratch;
    int sm_count;
    int blocks_per_sm[3];
};
constexpr int kMaxDevices = 64;
StaticDevice g_static_dev[kMaxDevices];
JumpTable g_static_unit;   // A^(2^k)
JumpTable g_static_chunk;  // A^(kStaticChunk 2^k)
bool g_static_tables = false;
std::mutex g_static_mu;

MatPair static_base()
{
    MatPair p;
    memset(&p, 0, sizeof p);
    uint32_t *a = p.a, *b = p.a + 9;
    a[1] = 1; a[5] = 1; a[6] = (uint32_t)(kM1 - 810728u); a[7] = 1403580u;
    b[1] = 1; b[5] = 1; b[6] = (uint32_t)(kM2 - 1370589u); b[8] = 527612u;
    return p;
}

srng_status static_setup(int dev, StaticDevice **out)
{
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_tables) {
        MatPair m = static_base();
        MatPair c = mat_identity(), sq = m;
        for (uint64_t e = kStaticChunk; e; e >>= 1) {  // A^kStaticChunk by square-and-multiply
            if (e & 1) c = mat_mul(c, sq);
            sq = mat_mul(sq, sq);
        }
        for (int k = 0; k < 64; ++k) {
            memcpy(g_static_unit.m[k], m.a, sizeof m.a);
            memcpy(g_static_chunk.m[k], c.a, sizeof c.a);
            m = mat_mul(m, m);
            c = mat_mul(c, c);
        }
        g_static_tables = true;
    }
    StaticDevice &d = g_static_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        SRNG_CUDA_TRY(cudaGetSymbolAddress(&p, g_batch_scratch));
        SRNG_CUDA_TRY(cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev));
        SRNG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.blocks_per_sm[0], k_batch_static<SRNG_OUT_U32>,
                                                                    kWarps * 32, 0));
        SRNG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.blocks_per_sm[1], k_batch_static<SRNG_OUT_F32>,
                                                                    kWarps * 32, 0));
        SRNG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.blocks_per_sm[2], k_batch_static<SRNG_OUT_F64>,
                                                                    kWarps * 32, 0));
        d.scratch = static_cast<unsigned char *>(p);
        d.ready = true;
    }
    *out = &d;
    return SRNG_OK;
}

}  // namespace
}  // namespace srng_impl

extern "C" srng_status srng_batch_run_static(srng_set *const *sets, uint32_t n_sets, const srng_instance *inst,
                                             uint64_t n_inst, srng_batch_mode mode, srng_out type, void *out_dev,
                                             void *cuda_stream)
{
    clear_error();
    if (mode != SRNG_BATCH_WRITE && mode != SRNG_BATCH_FUSED_PI) return fail(SRNG_ERR_ARG, "unknown batch mode");
    if (type != SRNG_OUT_U32 && type != SRNG_OUT_F32 && type != SRNG_OUT_F64)
        return fail(SRNG_ERR_ARG, "unknown output type");
    if (n_inst > kStaticMaxInst)
        return fail(SRNG_ERR_ARG, "srng_batch_run_static: more than SRNG_BATCH_STATIC_MAX_INSTANCES (4096) instances");
    if (n_sets > kStaticMaxSets)
        return fail(SRNG_ERR_ARG, "srng_batch_run_static: more than SRNG_BATCH_STATIC_MAX_SETS (8) sets");
    if (n_inst == 0) return SRNG_OK;
    if (!inst || !sets || n_sets == 0 || !out_dev) return fail(SRNG_ERR_ARG, "NULL instances, sets or output");
    const size_t esz = type == SRNG_OUT_F64 ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(out_dev) % (mode == SRNG_BATCH_WRITE ? esz : 8))
        return fail(SRNG_ERR_ARG, "output pointer misaligned");
    StaticSets ss;
    memset(&ss, 0, sizeof ss);
    for (uint32_t k = 0; k < n_sets; ++k) {
        const srng_set *s = sets[k];
        if (!s) return fail(SRNG_ERR_ARG, "NULL set");
        if (s->gen == SRNG_TINYMT32) return fail(SRNG_ERR_UNSUPPORTED, "TinyMT32 sets are not batched");
        ss.gen[k] = inst_gen(s);
        ss.key0[k] = s->key0;
        ss.key1[k] = s->key1;
        ss.keyed[k] = s->keyed ? 1u : 0u;
        ss.base[k] = s->stream_base;
        ss.state[k] = s->d_state;
        ss.ns[k] = s->n_streams;
        ss.pos[k] = s->d_pos;
    }
    // Work items per instance, counted as k_static_setup counts them: the
    // device side holds chunk indices, per-instance item numbers and the total
    // in 32-bit words, so calls that would overflow them are refused here,
    // before anything is enqueued.
    uint64_t total_items = 0;
    for (uint64_t i = 0; i < n_inst; ++i) {
        const srng_instance &x = inst[i];
        if (x.set_index >= n_sets) return fail(SRNG_ERR_ARG, "instance with a bad set index");
        const srng_set *s = sets[x.set_index];
        if (x.stream >= s->n_streams) return fail(SRNG_ERR_RANGE, "instance stream outside its set");
        if (x.length > (1ull << 48)) return fail(SRNG_ERR_ARG, "instance length above 2^48");
        if (s->gen == SRNG_PHILOX4X32_10 &&
            (x.offset > UINT64_MAX - s->max_pos || x.length > UINT64_MAX - s->max_pos - x.offset))
            return fail(SRNG_ERR_RANGE, "instance Philox position would pass 2^64 - 1");
        if (x.length == 0) continue;
        if (s->gen == SRNG_MRG32K3A) {
            const uint64_t nch = (x.length + kStaticChunk - 1) / kStaticChunk;
            if (nch > (1ull << 32))
                return fail(SRNG_ERR_ARG, "srng_batch_run_static: an MRG32k3a instance longer than 2^41 draws");
            total_items += (nch + 31) / 32;
        } else {
            const uint64_t nb = (x.length + 3) / 4 + 1, per = 32ull * kStaticLaneBlocks;
            total_items += (nb + per - 1) / per;
        }
        if (total_items > kStaticMaxItems)
            return fail(SRNG_ERR_ARG, "srng_batch_run_static: more than 2^31 work items in one call");
    }
    int dev = 0;
    SRNG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(SRNG_ERR_ARG, "device ordinal out of range");
    StaticDevice *d = nullptr;
    srng_status st = static_setup(dev, &d);
    if (st) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *scr = d->scratch;
    SRNG_CUDA_TRY(cudaMemcpyAsync(scr + kOffRaw, inst, n_inst * sizeof(srng_instance), cudaMemcpyHostToDevice, stream));
    const uint32_t n = (uint32_t)n_inst;
    k_static_setup<<<(n + 255) / 256, 256, 0, stream>>>(scr, n, ss, g_static_unit);
    SRNG_CUDA_TRY(cudaGetLastError());
    k_static_scan<<<1, 1024, 0, stream>>>(scr, n, mode == SRNG_BATCH_FUSED_PI ? static_cast<int64_t *>(out_dev)
                                                                              : nullptr);
    SRNG_CUDA_TRY(cudaGetLastError());
    BatchArgs a;
    memset(&a, 0, sizeof a);
    a.chunk = kStaticChunk;
    a.lane_blocks = kStaticLaneBlocks;
    a.mode = mode;
    a.out = out_dev;
    const unsigned grid = (unsigned)(d->sm_count * (d->blocks_per_sm[type] > 0 ? d->blocks_per_sm[type] : 1));
    switch (type) {
    case SRNG_OUT_U32: k_batch_static<SRNG_OUT_U32><<<grid, kWarps * 32, 0, stream>>>(scr, n, a, g_static_chunk); break;
    case SRNG_OUT_F32: k_batch_static<SRNG_OUT_F32><<<grid, kWarps * 32, 0, stream>>>(scr, n, a, g_static_chunk); break;
    default: k_batch_static<SRNG_OUT_F64><<<grid, kWarps * 32, 0, stream>>>(scr, n, a, g_static_chunk); break;
    }
    SRNG_CUDA_TRY(cudaGetLastError());
    return SRNG_OK;
}
