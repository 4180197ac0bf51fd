// K2 / K3 -- bulk generation with register-resident generator state, the
// fixed integer -> uniform conversion, and the output writer.
//
// K2 (MRG32k3a, paper Sec. 4.1): one thread owns a (stream, chunk) item.  It
// reaches the chunk's start state from the stream's state by jump-ahead
// (Sec. 2.3: chunk t starts at (A^C)^t y), then steps the recurrence in
// registers.  Because a thread's draws are contiguous in the stream-major
// output but 32 threads of a warp own 32 different rows, the warp stages a
// 32-row tile of 128-byte rows in shared memory and writes it back row by row
// (k_mrg_generate_rows: whole 128-byte lines per warp store; k_mrg_generate:
// 16-byte or element stores for any alignment), or, for whole-row items, each
// lane writes its own row with 32-byte stores straight from registers
// (k_mrg_generate_direct: one full sector per lane and store).
//
// K3 (Philox4x32-10, Threefry4x32-20 and Threefry4x64-20, Sec. 4.3):
// counter-based, so any position is computed directly.  A block of threads
// covers a contiguous run of 4-word groups of one stream (k_philox_generate):
// each lane writes its pair of groups -- eight values -- with 32-byte stores,
// so a warp store covers 1 KiB (u32 / f32); or the flat list of (stream, run
// of U block pairs) of many short streams (k_philox_generate_flat), each lane
// writing its run with 32-byte stores.
//
// Algorithmic HBM bytes per output value: the value's size (4 or 8); states
// and positions add 24 and 8 bytes per stream per call.
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "counter_based.cuh"
#include "internal.h"
#include "srng_device.cuh"

namespace srng_impl {

namespace {

template <int GEN, int OUT>
__device__ __forceinline__ typename OutType<OUT>::T convert(uint32_t v)
{
    if constexpr (OUT == SRNG_OUT_U32) return v;
    else if constexpr (OUT == SRNG_OUT_F32) return srng::to_f32(v);
    else if constexpr (OUT == SRNG_OUT_EXP_F32) return srng::dist::exponential(srng::to_f32(v));
    else if constexpr (GEN == SRNG_MRG32K3A) return srng::mrg::to_f64(v);
    else return srng::philox::to_f64(v);
}

// K output values from K consecutive words (K even).  The normal output pairs
// words (2i, 2i + 1) of the group (Box-Muller on their FP32 uniforms); every
// caller passes groups that start at an even draw of the stream (an even
// position for the counter-based generators, an even index of the call for
// the others).
template <int GEN, int OUT, int K>
__device__ __forceinline__ void convert_k(const uint32_t *w, typename OutType<OUT>::T *v)
{
    if constexpr (OUT == SRNG_OUT_NORMAL_F32) {
#pragma unroll
        for (int i = 0; i < K; i += 2) srng::dist::normal_pair(srng::to_f32(w[i]), srng::to_f32(w[i + 1]), &v[i], &v[i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i) v[i] = convert<GEN, OUT>(w[i]);
    }
}

// The state advance that follows an MRG32k3a generation launch is launched
// as its programmatic dependent: it may be scheduled once every block of the
// generation kernel has started, and it waits for the whole kernel to finish
// (and its memory to be visible) before it touches a state.
__device__ __forceinline__ void allow_dependent_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------------ K2
template <int OUT, bool VEC, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    k_mrg_generate(const MrgGenArgs a, const __grid_constant__ JumpTable tab)
{
    allow_dependent_launch();
    using T = typename OutType<OUT>::T;
    constexpr int G = 128 / sizeof(T);    // elements per 128-byte row (32 or 16)
    constexpr int VPL = 16 / sizeof(T);   // elements per 16-byte vector (4 or 2)
    constexpr int RS = G + VPL;           // row stride: 144 bytes, keeps 16-byte stores conflict-free
    __shared__ __align__(16) T tile[WARPS][32 * RS];
    __shared__ uint64_t row_off[WARPS][32];
    __shared__ uint32_t row_len[WARPS][32];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *my = &tile[warp][lane * RS];
    T *out = static_cast<T *>(a.out);
    const uint64_t n_items = a.s_count * a.cps;
    const uint64_t wstride = (uint64_t)gridDim.x * WARPS * 32;

    for (uint64_t base = ((uint64_t)blockIdx.x * WARPS + warp) * 32; base < n_items; base += wstride) {
        const uint64_t item = base + lane;
        uint64_t len = 0;
        uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
        if (item < n_items) {
            const uint64_t s_rel = item / a.cps;
            const uint64_t t = item - s_rel * a.cps;
            const uint64_t start = t * a.chunk;
            len = min(a.chunk, a.n - start);
            const uint64_t s = a.s_begin + s_rel;
            const uint64_t ns = a.n_streams;
            s0 = a.state[s]; s1 = a.state[ns + s]; s2 = a.state[2 * ns + s];
            s3 = a.state[3 * ns + s]; s4 = a.state[4 * ns + s]; s5 = a.state[5 * ns + s];
            for (int k = 0; k < a.nbits; ++k)
                if ((t >> k) & 1) srng::mrg::jump(tab.m[k], s0, s1, s2, s3, s4, s5);
            row_off[warp][lane] = s_rel * a.n + start;
        }
        const uint32_t ntiles = (uint32_t)((len + G - 1) / G);
        const uint32_t max_tiles = __reduce_max_sync(0xffffffffu, ntiles);

        for (uint32_t g = 0; g < max_tiles; ++g) {
            const uint64_t done = (uint64_t)g * G;
            const uint32_t rl = len > done ? (uint32_t)min((uint64_t)G, len - done) : 0u;
            row_len[warp][lane] = rl;
            for (uint32_t j = 0; j < rl; j += VPL) {
                if constexpr (sizeof(T) == 4) {
                    uint32_t w[4];
                    T x[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) w[e] = srng::mrg::step(s0, s1, s2, s3, s4, s5);
                    convert_k<SRNG_MRG32K3A, OUT, 4>(w, x);
                    *reinterpret_cast<uint4 *>(&my[j]) = *reinterpret_cast<const uint4 *>(x);
                } else {
                    double2 v;
                    v.x = convert<SRNG_MRG32K3A, OUT>(srng::mrg::step(s0, s1, s2, s3, s4, s5));
                    v.y = convert<SRNG_MRG32K3A, OUT>(srng::mrg::step(s0, s1, s2, s3, s4, s5));
                    *reinterpret_cast<double2 *>(&my[j]) = v;
                }
            }
            __syncwarp();
            constexpr int LPR = VEC ? G / VPL : G;  // lanes per row
            constexpr int RPI = 32 / LPR;           // rows per warp instruction
            const int q = lane % LPR, rsub = lane / LPR;
#pragma unroll 4
            for (int r0 = 0; r0 < 32; r0 += RPI) {
                const int r = r0 + rsub;
                const uint32_t rlen = row_len[warp][r];
                if constexpr (VEC) {
                    const uint32_t e = q * VPL;
                    if (e < rlen)
                        *reinterpret_cast<uint4 *>(out + row_off[warp][r] + done + e) =
                            *reinterpret_cast<const uint4 *>(&tile[warp][r * RS + e]);
                } else {
                    const uint32_t e = q;
                    if (e < rlen) out[row_off[warp][r] + done + e] = tile[warp][r * RS + e];
                }
            }
            __syncwarp();
        }
    }
}

// K2, uniform rows: every item is a whole chunk (n a multiple of chunk, chunk a
// multiple of the 128-byte row) and the output is 32-byte aligned, so item i's
// row starts at element i * chunk and every tile row is full.  Rows are written
// with 32-byte stores, four lanes per row, eight rows per warp instruction.
__device__ __forceinline__ void st256(void *p, uint4 a, uint4 b)
{
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a.x), "r"(a.y),
                 "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
                 : "memory");
}

template <int OUT, int WARPS, bool JUMP>
__global__ void __launch_bounds__(WARPS * 32)
    k_mrg_generate_rows(const MrgGenArgs a, const __grid_constant__ JumpTable tab)
{
    allow_dependent_launch();
    using T = typename OutType<OUT>::T;
    constexpr int G = 128 / sizeof(T);    // elements per 128-byte row
    constexpr int VPL = 16 / sizeof(T);   // elements per 16 bytes
    constexpr int RS = G + VPL;           // 144-byte row stride in shared memory
    constexpr int EPQ = 32 / sizeof(T);   // elements per 32-byte store
    __shared__ __align__(16) T tile[WARPS][32 * RS];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *my = &tile[warp][lane * RS];
    T *out = static_cast<T *>(a.out);
    const uint64_t n_items = a.s_count * a.cps;
    const uint64_t wstride = (uint64_t)gridDim.x * WARPS * 32;
    const int q = lane & 3, rsub = lane >> 2;

    for (uint64_t base = ((uint64_t)blockIdx.x * WARPS + warp) * 32; base < n_items; base += wstride) {
        const uint64_t item = base + lane;
        const bool active = item < n_items;
        const uint32_t rows = (uint32_t)min((uint64_t)32, n_items - base);
        uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
        if (active) {
            const uint64_t s_rel = JUMP ? item / a.cps : item;
            const uint64_t t = JUMP ? item - s_rel * a.cps : 0;
            const uint64_t s = a.s_begin + s_rel;
            const uint64_t ns = a.n_streams;
            s0 = a.state[s]; s1 = a.state[ns + s]; s2 = a.state[2 * ns + s];
            s3 = a.state[3 * ns + s]; s4 = a.state[4 * ns + s]; s5 = a.state[5 * ns + s];
            if (JUMP)
                for (int k = 0; k < a.nbits; ++k)
                    if ((t >> k) & 1) srng::mrg::jump(tab.m[k], s0, s1, s2, s3, s4, s5);
        }
        T *dst0 = out + base * a.chunk + (uint64_t)q * EPQ;
        for (uint64_t done = 0; done < a.chunk; done += G) {
            if (active) {
#pragma unroll
                for (int j = 0; j < G; j += VPL) {
                    if constexpr (sizeof(T) == 4) {
                        uint32_t w[4];
                        T x[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) w[e] = srng::mrg::step(s0, s1, s2, s3, s4, s5);
                        convert_k<SRNG_MRG32K3A, OUT, 4>(w, x);
                        *reinterpret_cast<uint4 *>(&my[j]) = *reinterpret_cast<uint4 *>(x);
                    } else {
                        double2 v;
                        v.x = convert<SRNG_MRG32K3A, OUT>(srng::mrg::step(s0, s1, s2, s3, s4, s5));
                        v.y = convert<SRNG_MRG32K3A, OUT>(srng::mrg::step(s0, s1, s2, s3, s4, s5));
                        *reinterpret_cast<double2 *>(&my[j]) = v;
                    }
                }
            }
            __syncwarp();
#pragma unroll
            for (int r0 = 0; r0 < 32; r0 += 8) {
                const int r = r0 + rsub;
                if ((uint32_t)r < rows) {
                    const T *src = &tile[warp][r * RS + q * EPQ];
                    st256(dst0 + (uint64_t)r * a.chunk + done, *reinterpret_cast<const uint4 *>(src),
                          *reinterpret_cast<const uint4 *>(src + VPL));
                }
            }
            __syncwarp();
        }
    }
}

// One lane's row of `chunk` values (a multiple of 8) from its registers, with
// 32-byte stores.  DMUL (FP64 only, a mask over each eight doubles): the doubles
// at its set positions come from the FP64 unit -- the multiply z * norm itself
// (the definition), or with FMA its one-instruction form (2^52 + z) norm -
// 2^52 norm -- and the others are built from integers, all the same bits, so
// the FP64 unit, otherwise idle, takes part of the conversions off the integer
// pipes.  The throughput-bound bulk rows take three in eight through the
// multiply (0x51: the 1st, 5th and 7th; one half makes the FP64 unit the
// bottleneck, and the FMA form measured slower there), the latency-bound rows
// of a few long streams one half through the FMA form (0x55).
constexpr uint32_t kDmulBulk = 0x51, kDmulLatency = 0x55;

template <int OUT, uint32_t DMUL, bool FMA = false>
__device__ __forceinline__ void lane_row(typename OutType<OUT>::T *dst, uint64_t chunk, uint32_t &s0, uint32_t &s1,
                                         uint32_t &s2, uint32_t &s3, uint32_t &s4, uint32_t &s5)
{
    using T = typename OutType<OUT>::T;
    constexpr int EPQ = 32 / sizeof(T);  // values per 32-byte store
    if constexpr (DMUL != 0 && OUT == SRNG_OUT_F64) {
        constexpr uint32_t kDmul = DMUL;
        for (uint64_t j = 0; j < chunk; j += 2 * EPQ) {
            uint32_t w[2 * EPQ];
            T v[2 * EPQ];
#pragma unroll
            for (int e = 0; e < 2 * EPQ; ++e) w[e] = srng::mrg::step(s0, s1, s2, s3, s4, s5);
#pragma unroll
            for (int e = 0; e < 2 * EPQ; ++e)
                v[e] = !((kDmul >> e) & 1) ? srng::mrg::to_f64(w[e])
                       : FMA                   ? srng::mrg::to_f64_fma(w[e])
                                               : srng::mrg::to_f64_dmul(w[e]);
            const uint4 *p = reinterpret_cast<const uint4 *>(v);
            st256(dst + j, p[0], p[1]);
            st256(dst + j + EPQ, p[2], p[3]);
        }
    } else {
        for (uint64_t j = 0; j < chunk; j += EPQ) {
            uint32_t w[EPQ];
            T v[EPQ];
#pragma unroll
            for (int e = 0; e < EPQ; ++e) w[e] = srng::mrg::step(s0, s1, s2, s3, s4, s5);
            convert_k<SRNG_MRG32K3A, OUT, EPQ>(w, v);
            const uint4 *p = reinterpret_cast<const uint4 *>(v);
            st256(dst + j, p[0], p[1]);
        }
    }
}

// K2, uniform rows, direct: each lane writes its own row with 32-byte stores
// straight from registers -- every store fills one whole 32-byte sector, 32
// sectors per warp instruction, no shared-memory transpose.  Same preconditions
// as k_mrg_generate_rows.  MIX: three in eight FP64 conversions on the FP64 unit
// (lane_row).
template <int OUT, int WARPS, bool JUMP, bool MIX = false>
__global__ void __launch_bounds__(WARPS * 32)
    k_mrg_generate_direct(const MrgGenArgs a, const __grid_constant__ JumpTable tab)
{
    allow_dependent_launch();
    using T = typename OutType<OUT>::T;
    T *out = static_cast<T *>(a.out);
    const uint64_t n_items = a.s_count * a.cps;
    const uint64_t stride = (uint64_t)gridDim.x * WARPS * 32;
    for (uint64_t item = (uint64_t)blockIdx.x * WARPS * 32 + threadIdx.x; item < n_items; item += stride) {
        const uint64_t s_rel = JUMP ? item / a.cps : item;
        const uint64_t t = JUMP ? item - s_rel * a.cps : 0;
        const uint64_t s = a.s_begin + s_rel;
        const uint64_t ns = a.n_streams;
        uint32_t s0 = a.state[s], s1 = a.state[ns + s], s2 = a.state[2 * ns + s];
        uint32_t s3 = a.state[3 * ns + s], s4 = a.state[4 * ns + s], s5 = a.state[5 * ns + s];
        if (JUMP)
            for (int k = 0; k < a.nbits; ++k)
                if ((t >> k) & 1) srng::mrg::jump(tab.m[k], s0, s1, s2, s3, s4, s5);
        lane_row<OUT, MIX ? kDmulBulk : 0u>(out + item * a.chunk, a.chunk, s0, s1, s2, s3, s4, s5);
    }
}

// Direct rows with radix-32 chunk starts, for streams cut into a multiple of
// 32 chunks: the 32 lanes of a warp take chunks t = 32 g + l (l the lane) of
// one stream, so that A^(C t) splits into A^(32 C (g mod 32)) -- the same
// matrix for the whole warp, read from the table in the parameters --,
// A^(C 2^k) for each set bit k >= 10 of t (also warp-uniform), and the lane's
// own A^(C l), read from a copy of the table in shared memory: at most two
// products for up to 1024 chunks per stream, where the bitwise jumps take one
// product per set bit of t and the warp waits for the slowest lane.  MIX: one
// half of the FP64 conversions as one FMA each on the FP64 unit (lane_row).
template <int OUT, int WARPS, bool MIX = false>
__global__ void __launch_bounds__(WARPS * 32)
    k_mrg_generate_radix(const MrgGenArgs a, const __grid_constant__ JumpTable tab,
                         const __grid_constant__ RadixTable rt)
{
    allow_dependent_launch();
    using T = typename OutType<OUT>::T;
    __shared__ __align__(16) uint32_t lane_m[32][20];  // 80-byte rows: conflict-free 16-byte reads
    for (int i = threadIdx.x; i < 32 * 18; i += WARPS * 32) lane_m[i / 18][i % 18] = rt.lane[i / 18][i % 18];
    __syncthreads();
    T *out = static_cast<T *>(a.out);
    const int lane = threadIdx.x & 31;
    const uint64_t n_items = a.s_count * a.cps;
    const uint64_t stride = (uint64_t)gridDim.x * WARPS * 32;
    for (uint64_t item = (uint64_t)blockIdx.x * WARPS * 32 + threadIdx.x; item < n_items; item += stride) {
        const uint64_t s_rel = item / a.cps;
        const uint64_t t = item - s_rel * a.cps;
        const uint64_t s = a.s_begin + s_rel;
        const uint64_t ns = a.n_streams;
        uint32_t s0 = a.state[s], s1 = a.state[ns + s], s2 = a.state[2 * ns + s];
        uint32_t s3 = a.state[3 * ns + s], s4 = a.state[4 * ns + s], s5 = a.state[5 * ns + s];
        const uint32_t g = (uint32_t)(t >> 5) & 31u;
        if (g) srng::mrg::jump(rt.warp[g], s0, s1, s2, s3, s4, s5);
        for (int k = 10; k < a.nbits; ++k)
            if ((t >> k) & 1) srng::mrg::jump(tab.m[k], s0, s1, s2, s3, s4, s5);
        if (lane) {
            uint32_t m[20];
            const uint4 *row = reinterpret_cast<const uint4 *>(lane_m[lane]);
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const uint4 v = row[q];
                m[4 * q] = v.x; m[4 * q + 1] = v.y; m[4 * q + 2] = v.z; m[4 * q + 3] = v.w;
            }
            srng::mrg::jump(m, s0, s1, s2, s3, s4, s5);
        }
        lane_row<OUT, MIX ? kDmulLatency : 0u, true>(out + item * a.chunk, a.chunk, s0, s1, s2, s3, s4, s5);
    }
}

// ------------------------------------------------------------------ K3
template <int GEN, int OUT, bool VEC>
__device__ __forceinline__ void store4(typename OutType<OUT>::T *row, int64_t k0, uint64_t n, const uint32_t *w)
{
    using T = typename OutType<OUT>::T;
    T vv[4];
    convert_k<GEN, OUT, 4>(w, vv);  // one block: its pairs are at even positions
    const T v0 = vv[0], v1 = vv[1], v2 = vv[2], v3 = vv[3];
    if (VEC && k0 >= 0 && (uint64_t)k0 + 4 <= n && ((reinterpret_cast<uintptr_t>(row + k0) & 15) == 0)) {
        if constexpr (sizeof(T) == 4) {
            uint4 v;
            v.x = *reinterpret_cast<const uint32_t *>(&v0);
            v.y = *reinterpret_cast<const uint32_t *>(&v1);
            v.z = *reinterpret_cast<const uint32_t *>(&v2);
            v.w = *reinterpret_cast<const uint32_t *>(&v3);
            *reinterpret_cast<uint4 *>(row + k0) = v;
        } else {
            *reinterpret_cast<double2 *>(row + k0) = make_double2(v0, v1);
            *reinterpret_cast<double2 *>(row + k0 + 2) = make_double2(v2, v3);
        }
    } else {
        const T v[4] = {v0, v1, v2, v3};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t k = k0 + j;
            if (k >= 0 && (uint64_t)k < n) row[k] = v[j];
        }
    }
}

// Eight consecutive output values (two Philox blocks) from one lane: one or two
// 32-byte stores when the run is inside the row and 32-byte aligned, else the
// 16-byte / element path of store4.
template <int GEN, int OUT, bool VEC>
__device__ __forceinline__ void store8(typename OutType<OUT>::T *row, int64_t k0, uint64_t n, const uint32_t *w)
{
    using T = typename OutType<OUT>::T;
    if (VEC && k0 >= 0 && (uint64_t)k0 + 8 <= n && ((reinterpret_cast<uintptr_t>(row + k0) & 31) == 0)) {
        T v[8];
        convert_k<GEN, OUT, 8>(w, v);
        const uint4 *p = reinterpret_cast<const uint4 *>(v);
        if constexpr (sizeof(T) == 4) {
            st256(row + k0, p[0], p[1]);
        } else {
            st256(row + k0, p[0], p[1]);
            st256(row + k0 + 4, p[2], p[3]);
        }
    } else {
        store4<GEN, OUT, VEC>(row, k0, n, w);
        store4<GEN, OUT, VEC>(row, k0 + 4, n, w + 4);
    }
}

// Tiles of 2 * blockDim.x * U Philox blocks; tps tiles per stream; the grid
// takes tiles by a stride of gridDim.x, tracked as (stream, tile) with the
// host's quotient / remainder of gridDim.x by tps.  Each lane computes U pairs
// of adjacent blocks (2U independent blocks in flight) and writes each pair's
// eight values with 32-byte stores: a warp store covers 1 KiB (u32 / f32).
// A tile lies wholly inside its stream's run when the stream's position is a
// multiple of the words per cipher block (no offset inside the first block)
// and the tile ends before the last whole block; such tiles of a 32-byte
// aligned row take a lean path (no bounds or alignment tests, FP32 through the
// conversion unit).  Every other tile takes the general path one pair at a
// time: partial pairs and misaligned runs with element stores.
template <int OUT, int U, bool VEC, int CIPHER>
__global__ void __launch_bounds__(256)
    k_philox_generate(const PhiloxGenArgs a, uint64_t tps, uint64_t q_grid, uint64_t r_grid)
{
    using T = typename OutType<OUT>::T;
    const uint64_t tb = 2ull * blockDim.x * U;
    const uint64_t n_tiles = a.s_count * tps;
    const uint64_t full = a.n / (4 * tb);  // whole tiles of a run that starts at a block boundary
    uint64_t s_rel = blockIdx.x / tps;
    uint64_t tt = blockIdx.x - s_rel * tps;
    uint64_t cur = ~0ull;  // stream whose position is loaded
    uint32_t al = 0, c2 = 0, c3 = 0, kk0 = a.k0, kk1 = a.k1;
    uint64_t q0 = 0, nb = 0;
    bool lean = false;
    T *row = nullptr;
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (s_rel != cur) {  // a block's tiles stay in one stream for long runs
            cur = s_rel;
            const uint64_t slot = a.s_begin + s_rel;
            const uint64_t p0 = a.pos[slot];
            const uint64_t s = a.stream_base + slot;  // stream number
            al = (uint32_t)p0 & cb_align_mask<CIPHER>();  // q0 even for Threefry4x64: one block per pair
            q0 = (p0 - al) >> 2;
            nb = (al + a.n + 3) >> 2;
            row = static_cast<T *>(a.out) + s_rel * a.n;
            lean = VEC && al == 0 && (reinterpret_cast<uintptr_t>(row) & 31) == 0;
            if (a.keyed) {  // key = the stream, counter words 2-3 = the seed
                kk0 = (uint32_t)s; kk1 = (uint32_t)(s >> 32); c2 = a.k0; c3 = a.k1;
            } else {
                c2 = (uint32_t)s; c3 = (uint32_t)(s >> 32);
            }
        }
        if (lean && tt < full) {
            uint32_t x[U][8];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t b = tt * tb + (uint64_t)u * 2 * blockDim.x + 2 * threadIdx.x;
                cb_pair<CIPHER, true>(q0 + b, x[u], kk0, kk1, c2, c3);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t b = tt * tb + (uint64_t)u * 2 * blockDim.x + 2 * threadIdx.x;
                T v[8];
                if constexpr (OUT == SRNG_OUT_F32) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = srng::to_f32_cvt(x[u][j]);
                } else {
                    convert_k<SRNG_PHILOX4X32_10, OUT, 8>(x[u], v);
                }
                const uint4 *p = reinterpret_cast<const uint4 *>(v);
                st256(row + 4 * b, p[0], p[1]);
                if constexpr (sizeof(T) == 8) st256(row + 4 * b + 4, p[2], p[3]);
            }
        } else {
#pragma unroll 1
            for (int u = 0; u < U; ++u) {
                const uint64_t b = tt * tb + (uint64_t)u * 2 * blockDim.x + 2 * threadIdx.x;
                if (b >= nb) break;
                uint32_t w[8];
                cb_pair<CIPHER, true>(q0 + b, w, kk0, kk1, c2, c3);
                store8<SRNG_PHILOX4X32_10, OUT, VEC>(row, (int64_t)(b * 4) - al, a.n, w);
            }
        }
        tt += r_grid;
        s_rel += q_grid;
        if (tt >= tps) { tt -= tps; ++s_rel; }
    }
}

// Division by an invariant 32-bit d (Granlund & Montgomery, PLDI 1994): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, for every 32-bit n,
// t = umulhi(m, n) and n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
struct Divider {
    uint32_t d, m;
    uint32_t sh1, sh2;
};

inline Divider make_divider(uint32_t d)
{
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    Divider v;
    v.d = d;
    v.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    v.sh1 = l < 1 ? l : 1;
    v.sh2 = l > 1 ? l - 1 : 0;
    return v;
}

__device__ __forceinline__ uint32_t divide(uint32_t n, const Divider &v)
{
    const uint32_t t = __umulhi(v.m, n);
    return (t + ((n - t) >> v.sh1)) >> v.sh2;
}

// Flat Philox generation for many short streams: the work is the flat list of
// (stream, group) with gps groups per stream, a group being U consecutive block
// pairs of one stream, so that the division of the group index, the stream's
// position load and its key or counter words are paid once per U pairs (the
// key-per-stream layout gains most); no lane idles at a stream's end beyond
// its last group.  Every store is a full 32-byte sector.
template <int OUT, int U, bool VEC, int CIPHER>
__global__ void __launch_bounds__(256)
    k_philox_generate_flat(const PhiloxGenArgs a, uint32_t total_groups, const Divider gps)
{
    using T = typename OutType<OUT>::T;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total_groups; g += stride) {
        const uint32_t s_rel = divide(g, gps);
        const uint64_t b0 = 2ull * U * (g - s_rel * gps.d);  // first block of the group
        const uint64_t slot = a.s_begin + s_rel;
        const uint64_t pos = a.pos[slot];
        const uint32_t al = (uint32_t)pos & cb_align_mask<CIPHER>();
        const uint64_t nb = (al + a.n + 3) >> 2;
        const uint64_t s = a.stream_base + slot;
        uint32_t kk0 = a.k0, kk1 = a.k1, c2, c3;
        if (a.keyed) { kk0 = (uint32_t)s; kk1 = (uint32_t)(s >> 32); c2 = a.k0; c3 = a.k1; }
        else { c2 = (uint32_t)s; c3 = (uint32_t)(s >> 32); }
        const uint64_t q0 = (pos - al) >> 2;
        T *row = static_cast<T *>(a.out) + (uint64_t)s_rel * a.n;
        uint32_t x[U][8];
#pragma unroll
        for (int u = 0; u < U; ++u) cb_pair<CIPHER, true>(q0 + b0 + 2 * u, x[u], kk0, kk1, c2, c3);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (b0 + 2 * u < nb) store8<SRNG_PHILOX4X32_10, OUT, VEC>(row, (int64_t)((b0 + 2 * u) * 4) - al, a.n, x[u]);
    }
}

// ---------------------------------------------------------- variates
// Exponential: out[i] = -ln(1 - in[i]); normal: Box-Muller on the pairs
// (in[2k], in[2k+1]).  Elementwise, 4 bytes read and 4 written per value:
// HBM bound (normal: close to the FP32 pipe as well).  Each block takes
// contiguous tiles of 1024 float4, four 16-byte loads in flight per thread;
// the n mod 4 tail goes scalar.
template <int DIST> __device__ __forceinline__ float4 variates4(float4 u)
{
    float4 v;
    if (DIST == SRNG_DIST_EXPONENTIAL) {
        v.x = srng::dist::exponential(u.x); v.y = srng::dist::exponential(u.y);
        v.z = srng::dist::exponential(u.z); v.w = srng::dist::exponential(u.w);
    } else {
        srng::dist::normal_pair(u.x, u.y, &v.x, &v.y);
        srng::dist::normal_pair(u.z, u.w, &v.z, &v.w);
    }
    return v;
}

constexpr int kTransformU = 2;  // float4 per thread per trip of k_transform (1: slower, 4 without prefetch: slower)

template <int DIST>
__global__ void __launch_bounds__(256) k_transform(const float *in, uint64_t n, float *out)  // in == out allowed
{
    constexpr int U = kTransformU;
    constexpr uint64_t kTile = 256 * U;       // float4 per block per trip, contiguous
    const uint64_t n4 = n / 4;
    const uint64_t step = (uint64_t)gridDim.x * kTile;
    const float4 *in4 = reinterpret_cast<const float4 *>(in);
    float4 *out4 = reinterpret_cast<float4 *>(out);
    // the next trip's loads are issued before this trip's arithmetic (trips
    // touch disjoint elements, so in == out stays allowed)
    float4 a[U];
    uint64_t base = (uint64_t)blockIdx.x * kTile;
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const uint64_t i = base + k * 256 + threadIdx.x;
        if (i < n4) a[k] = in4[i];
    }
    for (; base < n4; base += step) {
        float4 nx[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint64_t i = base + step + k * 256 + threadIdx.x;
            if (i < n4) nx[k] = in4[i];
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint64_t i = base + k * 256 + threadIdx.x;
            if (i < n4) out4[i] = variates4<DIST>(a[k]);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) a[k] = nx[k];
    }
    if (blockIdx.x == 0) {                    // the n mod 4 tail
        const uint64_t t = 4 * n4 + (DIST == SRNG_DIST_EXPONENTIAL ? threadIdx.x : 2 * threadIdx.x);
        if (DIST == SRNG_DIST_EXPONENTIAL) {
            if (t < n) out[t] = srng::dist::exponential(in[t]);
        } else if (t + 1 < n) {
            float z0, z1;
            srng::dist::normal_pair(in[t], in[t + 1], &z0, &z1);
            out[t] = z0;
            out[t + 1] = z1;
        }
    }
}

// Pointers not 16-byte aligned: one value (exponential) or pair (normal) per step.
template <int DIST>
__global__ void __launch_bounds__(256) k_transform_scalar(const float *in, uint64_t n, float *out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (DIST == SRNG_DIST_NORMAL ? n / 2 : n);
         i += stride) {
        if (DIST == SRNG_DIST_EXPONENTIAL) {
            out[i] = srng::dist::exponential(in[i]);
        } else {
            float z0, z1;
            srng::dist::normal_pair(in[2 * i], in[2 * i + 1], &z0, &z1);
            out[2 * i] = z0;
            out[2 * i + 1] = z1;
        }
    }
}

// ---------------------------------------------------------- conversion
template <int GEN, int OUT>
__global__ void __launch_bounds__(256) k_convert(const uint32_t *__restrict__ in, uint64_t n,
                                                 typename OutType<OUT>::T *__restrict__ out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = convert<GEN, OUT>(in[i]);
}

template <int OUT, bool VEC>
cudaError_t mrg_dispatch_warps(const MrgGenArgs &a, const JumpTable &tab, const srng_tune &t,
                               cudaStream_t stream, const DeviceInfo &dev)
{
    const uint64_t items = a.s_count * a.cps;
    const int warps = t.block_threads >= 256 ? 8 : 4;
    uint64_t blocks = (items + warps * 32 - 1) / (warps * 32);
    uint64_t cap = (uint64_t)dev.sm_count * (t.blocks_per_sm ? t.blocks_per_sm : 5);
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    if (warps == 8) k_mrg_generate<OUT, VEC, 8><<<(unsigned)blocks, 256, 0, stream>>>(a, tab);
    else k_mrg_generate<OUT, VEC, 4><<<(unsigned)blocks, 128, 0, stream>>>(a, tab);
    return cudaGetLastError();
}

// Dynamic shared memory that holds kernel k to at most `resident` blocks per SM
// (0: no limit, or none needed), found from the SM's shared memory and checked
// with the occupancy calculator; cached per (kernel, threads, limit, device).
template <typename K>
size_t residency_smem(K k, int threads, uint32_t resident)
{
    if (!resident) return 0;
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, uint32_t, int>, size_t> cache;
    std::lock_guard<std::mutex> lk(mu);
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(reinterpret_cast<const void *>(k), threads, resident, dev);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    size_t dyn = 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, 0) == cudaSuccess && nb > (int)resident) {
        int per_sm = 0, reserved = 0;
        cudaFuncAttributes fa;
        if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, k) == cudaSuccess) {
            const long want = (long)per_sm / (long)resident - reserved - (long)fa.sharedSizeBytes;
            if (want > 0) {
                dyn = (size_t)want;
                // static + dynamic above 48 KiB needs the kernel's opt-in
                auto allow = [&]() {
                    if (fa.sharedSizeBytes + dyn > 48 * 1024)
                        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
                };
                allow();
                // never more than `resident`: grow the reservation until the calculator agrees
                for (int step = 0; step < 64; ++step) {
                    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, dyn) != cudaSuccess) break;
                    if (nb <= (int)resident) break;
                    dyn += 256;
                    allow();
                }
            }
        }
        cudaGetLastError();  // a refused attribute leaves no error behind; the launch then runs unlimited
    }
    cache.emplace(key, dyn);
    return dyn;
}

template <typename K>
void launch_limited(K k, unsigned grid, int threads, const srng_tune &t, cudaStream_t stream, const MrgGenArgs &a,
                    const JumpTable &tab)
{
    k<<<grid, threads, residency_smem(k, threads, t.resident), stream>>>(a, tab);
}

template <typename K>
void launch_limited(K k, unsigned grid, int threads, const srng_tune &t, cudaStream_t stream, const MrgGenArgs &a,
                    const JumpTable &tab, const RadixTable &rt)
{
    k<<<grid, threads, residency_smem(k, threads, t.resident), stream>>>(a, tab, rt);
}

template <int OUT>
cudaError_t mrg_dispatch_rows(const MrgGenArgs &a, const JumpTable &tab, const srng_tune &t, cudaStream_t stream,
                              const DeviceInfo &dev, const RadixTable *rt)
{
    const uint64_t items = a.s_count * a.cps;
    const int warps = t.block_threads >= 256 ? 8 : 4;
    uint64_t blocks = (items + warps * 32 - 1) / (warps * 32);
    uint64_t cap = (uint64_t)dev.sm_count * (t.blocks_per_sm ? t.blocks_per_sm : 5);
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    // one item per stream (no chunk starts to reach): kernels without the jump code
    const bool jump = a.cps > 1;
    const unsigned g = (unsigned)blocks;
    if (rt && jump && a.cps % 32 == 0 && (t.vector_store == 3 || t.vector_store == 4)) {
        constexpr bool F64 = OUT == SRNG_OUT_F64;  // the mixed conversion exists for doubles only
        const bool mix = F64 && t.vector_store == 4;
        if (warps == 8) {
            if (mix) launch_limited(k_mrg_generate_radix<OUT, 8, F64>, g, 256, t, stream, a, tab, *rt);
            else launch_limited(k_mrg_generate_radix<OUT, 8, false>, g, 256, t, stream, a, tab, *rt);
        } else {
            if (mix) launch_limited(k_mrg_generate_radix<OUT, 4, F64>, g, 128, t, stream, a, tab, *rt);
            else launch_limited(k_mrg_generate_radix<OUT, 4, false>, g, 128, t, stream, a, tab, *rt);
        }
        return cudaGetLastError();
    }
    if constexpr (OUT == SRNG_OUT_F64) {
        if (t.vector_store == 4) {  // direct rows, three in eight doubles through the FP64 multiply
            if (warps == 8) {
                if (jump) launch_limited(k_mrg_generate_direct<OUT, 8, true, true>, g, 256, t, stream, a, tab);
                else launch_limited(k_mrg_generate_direct<OUT, 8, false, true>, g, 256, t, stream, a, tab);
            } else {
                if (jump) launch_limited(k_mrg_generate_direct<OUT, 4, true, true>, g, 128, t, stream, a, tab);
                else launch_limited(k_mrg_generate_direct<OUT, 4, false, true>, g, 128, t, stream, a, tab);
            }
            return cudaGetLastError();
        }
    }
    if (t.vector_store == 3 || t.vector_store == 4) {
        if (warps == 8) {
            if (jump) launch_limited(k_mrg_generate_direct<OUT, 8, true>, g, 256, t, stream, a, tab);
            else launch_limited(k_mrg_generate_direct<OUT, 8, false>, g, 256, t, stream, a, tab);
        } else {
            if (jump) launch_limited(k_mrg_generate_direct<OUT, 4, true>, g, 128, t, stream, a, tab);
            else launch_limited(k_mrg_generate_direct<OUT, 4, false>, g, 128, t, stream, a, tab);
        }
    } else {
        if (warps == 8) {
            if (jump) launch_limited(k_mrg_generate_rows<OUT, 8, true>, g, 256, t, stream, a, tab);
            else launch_limited(k_mrg_generate_rows<OUT, 8, false>, g, 256, t, stream, a, tab);
        } else {
            if (jump) launch_limited(k_mrg_generate_rows<OUT, 4, true>, g, 128, t, stream, a, tab);
            else launch_limited(k_mrg_generate_rows<OUT, 4, false>, g, 128, t, stream, a, tab);
        }
    }
    return cudaGetLastError();
}

template <int OUT>
cudaError_t mrg_dispatch(const MrgGenArgs &a, const JumpTable &tab, const srng_tune &t, cudaStream_t stream,
                         const DeviceInfo &dev, const RadixTable *rt)
{
    using T = typename OutType<OUT>::T;
    constexpr uint64_t VPL = 16 / sizeof(T);
    constexpr uint64_t G = 128 / sizeof(T);
    if (t.vector_store != 2 && (reinterpret_cast<uintptr_t>(a.out) & 31) == 0 && a.n % a.chunk == 0 &&
        a.chunk % G == 0)
        return mrg_dispatch_rows<OUT>(a, tab, t, stream, dev, rt);
    const bool vec_ok = t.vector_store != 2 && (reinterpret_cast<uintptr_t>(a.out) & 15) == 0 &&
                        a.n % VPL == 0 && a.chunk % VPL == 0;
    return vec_ok ? mrg_dispatch_warps<OUT, true>(a, tab, t, stream, dev)
                  : mrg_dispatch_warps<OUT, false>(a, tab, t, stream, dev);
}

template <int OUT, int U, int CIPHER>
cudaError_t philox_dispatch_u(const PhiloxGenArgs &a, const srng_tune &t, cudaStream_t stream,
                              const DeviceInfo &dev)
{
    const uint32_t threads = t.block_threads ? t.block_threads : 256;
    const uint64_t bps = (a.n + cb_align_mask<CIPHER>() + 3) / 4;  // blocks per stream, any start offset
    const uint64_t tb = 2ull * threads * U;
    const uint64_t tps = (bps + tb - 1) / tb;
    const uint64_t n_tiles = a.s_count * tps;
    uint64_t blocks = n_tiles;
    const uint64_t cap = (uint64_t)dev.sm_count * (t.blocks_per_sm ? t.blocks_per_sm : 2048 / threads);
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    const uint64_t qg = blocks / tps, rg = blocks % tps;
    if (t.vector_store != 2)
        k_philox_generate<OUT, U, true, CIPHER><<<(unsigned)blocks, threads, 0, stream>>>(a, tps, qg, rg);
    else
        k_philox_generate<OUT, U, false, CIPHER><<<(unsigned)blocks, threads, 0, stream>>>(a, tps, qg, rg);
    return cudaGetLastError();
}

template <int OUT, int CIPHER>
cudaError_t philox_dispatch(const PhiloxGenArgs &a, const srng_tune &t, cudaStream_t stream, const DeviceInfo &dev)
{
    // Many short streams: the flat kernel (no idle lanes at stream ends), when
    // a stream is shorter than one tile and the pair count stays below 2^31 (so
    // the kernel's 32-bit group index plus its grid stride, below 2^22, cannot
    // wrap).
    const uint64_t pps = ((a.n + cb_align_mask<CIPHER>() + 3) / 4 + 1) / 2;  // block pairs per stream, any start offset
    const uint32_t threads = t.block_threads ? t.block_threads : 256;
    const uint64_t tile_pairs = (uint64_t)threads * (t.unroll ? t.unroll : 4);
    if (a.s_count > 1 && pps < tile_pairs && a.s_count * pps < (1ull << 31)) {
        const uint32_t uu = t.unroll == 1 ? 1u : t.unroll == 4 ? 4u : 2u;  // pairs per group (the kernel's U)
        const uint64_t gps = (pps + uu - 1) / uu;                             // groups per stream
        const uint32_t total = (uint32_t)(a.s_count * gps);
        uint64_t blocks = (total + threads - 1) / threads;
        const uint64_t cap = (uint64_t)dev.sm_count * (t.blocks_per_sm ? t.blocks_per_sm : 2048 / threads);
        if (blocks > cap) blocks = cap;
        const Divider dv = make_divider((uint32_t)gps);
        const bool vec = t.vector_store != 2;
        if (t.unroll == 1) {
            if (vec) k_philox_generate_flat<OUT, 1, true, CIPHER><<<(unsigned)blocks, threads, 0, stream>>>(a, total, dv);
            else k_philox_generate_flat<OUT, 1, false, CIPHER><<<(unsigned)blocks, threads, 0, stream>>>(a, total, dv);
        } else if (t.unroll == 4) {
            if (vec) k_philox_generate_flat<OUT, 4, true, CIPHER><<<(unsigned)blocks, threads, 0, stream>>>(a, total, dv);
            else k_philox_generate_flat<OUT, 4, false, CIPHER><<<(unsigned)blocks, threads, 0, stream>>>(a, total, dv);
        } else {
            if (vec) k_philox_generate_flat<OUT, 2, true, CIPHER><<<(unsigned)blocks, threads, 0, stream>>>(a, total, dv);
            else k_philox_generate_flat<OUT, 2, false, CIPHER><<<(unsigned)blocks, threads, 0, stream>>>(a, total, dv);
        }
        return cudaGetLastError();
    }
    switch (t.unroll) {
    case 1: return philox_dispatch_u<OUT, 1, CIPHER>(a, t, stream, dev);
    case 4: return philox_dispatch_u<OUT, 4, CIPHER>(a, t, stream, dev);
    default: return philox_dispatch_u<OUT, 2, CIPHER>(a, t, stream, dev);
    }
}

}  // namespace

cudaError_t launch_mrg_generate(const MrgGenArgs &a, srng_out type, const JumpTable &tab, const srng_tune &t,
                                cudaStream_t stream, const DeviceInfo &dev, const RadixTable *rt)
{
    switch (type) {
    case SRNG_OUT_U32: return mrg_dispatch<SRNG_OUT_U32>(a, tab, t, stream, dev, rt);
    case SRNG_OUT_F32: return mrg_dispatch<SRNG_OUT_F32>(a, tab, t, stream, dev, rt);
    case SRNG_OUT_EXP_F32: return mrg_dispatch<SRNG_OUT_EXP_F32>(a, tab, t, stream, dev, rt);
    case SRNG_OUT_NORMAL_F32: return mrg_dispatch<SRNG_OUT_NORMAL_F32>(a, tab, t, stream, dev, rt);
    default: return mrg_dispatch<SRNG_OUT_F64>(a, tab, t, stream, dev, rt);
    }
}

cudaError_t launch_philox_generate(const PhiloxGenArgs &a, srng_out type, const srng_tune &t,
                                   cudaStream_t stream, const DeviceInfo &dev)
{
    if (a.threefry == 2) {
        switch (type) {
        case SRNG_OUT_U32: return philox_dispatch<SRNG_OUT_U32, kCipherThreefry64>(a, t, stream, dev);
        case SRNG_OUT_F32: return philox_dispatch<SRNG_OUT_F32, kCipherThreefry64>(a, t, stream, dev);
        case SRNG_OUT_EXP_F32: return philox_dispatch<SRNG_OUT_EXP_F32, kCipherThreefry64>(a, t, stream, dev);
        case SRNG_OUT_NORMAL_F32: return philox_dispatch<SRNG_OUT_NORMAL_F32, kCipherThreefry64>(a, t, stream, dev);
        default: return philox_dispatch<SRNG_OUT_F64, kCipherThreefry64>(a, t, stream, dev);
        }
    }
    if (a.threefry) {
        switch (type) {
        case SRNG_OUT_U32: return philox_dispatch<SRNG_OUT_U32, kCipherThreefry>(a, t, stream, dev);
        case SRNG_OUT_F32: return philox_dispatch<SRNG_OUT_F32, kCipherThreefry>(a, t, stream, dev);
        case SRNG_OUT_EXP_F32: return philox_dispatch<SRNG_OUT_EXP_F32, kCipherThreefry>(a, t, stream, dev);
        case SRNG_OUT_NORMAL_F32: return philox_dispatch<SRNG_OUT_NORMAL_F32, kCipherThreefry>(a, t, stream, dev);
        default: return philox_dispatch<SRNG_OUT_F64, kCipherThreefry>(a, t, stream, dev);
        }
    }
    switch (type) {
    case SRNG_OUT_U32: return philox_dispatch<SRNG_OUT_U32, kCipherPhilox>(a, t, stream, dev);
    case SRNG_OUT_F32: return philox_dispatch<SRNG_OUT_F32, kCipherPhilox>(a, t, stream, dev);
    case SRNG_OUT_EXP_F32: return philox_dispatch<SRNG_OUT_EXP_F32, kCipherPhilox>(a, t, stream, dev);
    case SRNG_OUT_NORMAL_F32: return philox_dispatch<SRNG_OUT_NORMAL_F32, kCipherPhilox>(a, t, stream, dev);
    default: return philox_dispatch<SRNG_OUT_F64, kCipherPhilox>(a, t, stream, dev);
    }
}

cudaError_t launch_transform(int dist, const float *in, uint64_t n, float *out, cudaStream_t stream,
                             const DeviceInfo &dev)
{
    if (n == 0) return cudaSuccess;
    // resident blocks per SM: 4 for the exponential (memory bound), 8 for the
    // normal (more arithmetic to hide); measured on GB300 at 2^30 values
    const uint64_t cap = (uint64_t)dev.sm_count * (dist == SRNG_DIST_NORMAL ? 8 : 4);
    const bool vec = (reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % 16 == 0;
    uint64_t blocks = vec ? (n / 4 + 256 * kTransformU - 1) / (256 * kTransformU) : (n + 255) / 256;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;   // the scalar tail of a short input
    const unsigned g = (unsigned)blocks;
    if (vec) {
        if (dist == SRNG_DIST_EXPONENTIAL) k_transform<SRNG_DIST_EXPONENTIAL><<<g, 256, 0, stream>>>(in, n, out);
        else k_transform<SRNG_DIST_NORMAL><<<g, 256, 0, stream>>>(in, n, out);
    } else {
        if (dist == SRNG_DIST_EXPONENTIAL) k_transform_scalar<SRNG_DIST_EXPONENTIAL><<<g, 256, 0, stream>>>(in, n, out);
        else k_transform_scalar<SRNG_DIST_NORMAL><<<g, 256, 0, stream>>>(in, n, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_convert(srng_gen gen, srng_out type, const uint32_t *in, uint64_t n, void *out,
                           cudaStream_t stream, const DeviceInfo &dev)
{
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    const uint64_t cap = (uint64_t)dev.sm_count * 8;
    if (blocks > cap) blocks = cap;
    const unsigned g = (unsigned)blocks;
    if (gen == SRNG_MRG32K3A) {
        if (type == SRNG_OUT_U32) k_convert<SRNG_MRG32K3A, SRNG_OUT_U32><<<g, 256, 0, stream>>>(in, n, (uint32_t *)out);
        else if (type == SRNG_OUT_F32) k_convert<SRNG_MRG32K3A, SRNG_OUT_F32><<<g, 256, 0, stream>>>(in, n, (float *)out);
        else k_convert<SRNG_MRG32K3A, SRNG_OUT_F64><<<g, 256, 0, stream>>>(in, n, (double *)out);
    } else {
        if (type == SRNG_OUT_U32) k_convert<SRNG_PHILOX4X32_10, SRNG_OUT_U32><<<g, 256, 0, stream>>>(in, n, (uint32_t *)out);
        else if (type == SRNG_OUT_F32) k_convert<SRNG_PHILOX4X32_10, SRNG_OUT_F32><<<g, 256, 0, stream>>>(in, n, (float *)out);
        else k_convert<SRNG_PHILOX4X32_10, SRNG_OUT_F64><<<g, 256, 0, stream>>>(in, n, (double *)out);
    }
    return cudaGetLastError();
}

}  // namespace srng_impl
