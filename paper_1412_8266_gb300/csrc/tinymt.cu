// K8 -- TinyMT32 (paper Sec. 4.2): the hybrid partition of parameterised
// statuses.  A parameter set (mat1, mat2, tmat) serves a group of streams --
// the threads of a CUDA block in the paper -- and the streams of a group are
// substreams of the group's sequence, 2^64 steps apart (sequence splitting).
//
// Jumps: the step T is GF(2)-linear with characteristic polynomial p of
// degree 127, so T^J s = r(T) s with r = x^J mod p.  The host computes r per
// parameter set; a device thread evaluates r(T) s by Horner's rule (127 steps
// with a masked xor of s), about 2,000 integer instructions.
//
//   k_tmt_place     stream i of group g: T^(j 2^64) seed_g, j = i mod group
//                   size, one Horner jump per set bit of j
//   k_tmt_apply     state <- r_g(T) state (srng_jump, state advance)
//   k_tmt_generate  item = (stream, chunk t); the chunk's start by Horner
//                   jumps x^(chunk 2^k) for the set bits of t; each lane then
//                   writes its own row segment with 32-byte stores from
//                   registers (element stores at an unaligned head or tail)
//
// Algorithmic HBM bytes per value: its size (4 or 8); 16 bytes of state per
// stream per call.
#include <stdint.h>

#include "internal.h"
#include "srng_device.cuh"

namespace srng_impl {

namespace {

constexpr int kThreads = 256;

template <int OUT> __device__ __forceinline__ typename OutType<OUT>::T tconv(uint32_t v)
{
    if constexpr (OUT == SRNG_OUT_U32) return v;
    else if constexpr (OUT == SRNG_OUT_F32) return srng::to_f32(v);
    else if constexpr (OUT == SRNG_OUT_EXP_F32) return srng::dist::exponential(srng::to_f32(v));
    else return srng::philox::to_f64(v);
}

__device__ __forceinline__ void tst256(void *p, const uint32_t *w)
{
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

__global__ void __launch_bounds__(kThreads)
    k_tmt_place(uint32_t *__restrict__ st, uint64_t ns, const uint4 *__restrict__ params, uint64_t gs,
                const uint4 *__restrict__ seeds, const uint4 *__restrict__ jt, int nbits)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += stride) {
        const uint64_t g = i / gs, j = i - g * gs;
        const uint4 p = params[g], sd = seeds[g];
        uint32_t s0 = sd.x, s1 = sd.y, s2 = sd.z, s3 = sd.w;
        for (int k = 0; k < nbits; ++k)
            if ((j >> k) & 1) srng::tinymt::jump(jt[g * nbits + k], s0, s1, s2, s3, p.x, p.y);
        st[i] = s0; st[ns + i] = s1; st[2 * ns + i] = s2; st[3 * ns + i] = s3;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_tmt_apply(uint32_t *__restrict__ st, uint64_t ns, const uint4 *__restrict__ params, uint64_t gs,
                uint64_t first, uint64_t count, const uint4 *__restrict__ poly, uint64_t g0)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += stride) {
        const uint64_t i = first + r, g = i / gs;
        const uint4 p = params[g];
        uint32_t s0 = st[i], s1 = st[ns + i], s2 = st[2 * ns + i], s3 = st[3 * ns + i];
        srng::tinymt::jump(poly[g - g0], s0, s1, s2, s3, p.x, p.y);
        st[i] = s0; st[ns + i] = s1; st[2 * ns + i] = s2; st[3 * ns + i] = s3;
    }
}

template <int OUT>
__global__ void __launch_bounds__(kThreads) k_tmt_generate(const TmtGenArgs a)
{
    using T = typename OutType<OUT>::T;
    constexpr int EPQ = 32 / sizeof(T);  // values per 32-byte store
    const uint64_t n_items = a.s_count * a.cps;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t ns = a.n_streams;
    for (uint64_t item = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; item < n_items; item += stride) {
        const uint64_t s_rel = item / a.cps, t = item - s_rel * a.cps;
        const uint64_t s = a.s_begin + s_rel, g = s / a.group_size;
        const uint4 p = a.params[g];
        uint32_t s0 = a.state[s], s1 = a.state[ns + s], s2 = a.state[2 * ns + s], s3 = a.state[3 * ns + s];
        for (int k = 0; k < a.nbits; ++k)
            if ((t >> k) & 1) srng::tinymt::jump(a.jtab[(g - a.g0) * a.nbits + k], s0, s1, s2, s3, p.x, p.y);
        const uint64_t k0 = t * a.chunk;
        const uint64_t len = min(a.chunk, a.n - k0);
        T *row = static_cast<T *>(a.out) + s_rel * a.n + k0;
        if constexpr (OUT == SRNG_OUT_NORMAL_F32) {
            // pairs of draws (2i, 2i + 1) of the item (the chunk and n are even):
            // groups of eight values, 32-byte stores when aligned
            for (uint64_t done = 0; done < len; done += 8) {
                const uint32_t cnt = (uint32_t)min((uint64_t)8, len - done);
                uint32_t w[8];
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    if ((uint32_t)e < cnt) srng::tinymt::step(s0, s1, s2, s3, p.x, p.y);
                    w[e] = srng::tinymt::temper(s0, s2, s3, p.z);
                }
#pragma unroll
                for (int e = 0; e < 8; e += 2)
                    srng::dist::normal_pair(srng::to_f32(w[e]), srng::to_f32(w[e + 1]), &v[e], &v[e + 1]);
                if (cnt == 8 && (reinterpret_cast<uintptr_t>(row + done) & 31u) == 0) {
                    tst256(row + done, reinterpret_cast<const uint32_t *>(v));
                } else {
                    for (uint32_t e = 0; e < cnt; ++e) row[done + e] = v[e];
                }
            }
            if (a.write_back) {
                a.state[s] = s0; a.state[ns + s] = s1; a.state[2 * ns + s] = s2; a.state[3 * ns + s] = s3;
            }
            continue;
        }
        uint64_t head = ((32u - (reinterpret_cast<uintptr_t>(row) & 31u)) & 31u) / sizeof(T);
        if (head > len) head = len;
        uint64_t done = 0;
        for (; done < head; ++done) {
            srng::tinymt::step(s0, s1, s2, s3, p.x, p.y);
            row[done] = tconv<OUT>(srng::tinymt::temper(s0, s2, s3, p.z));
        }
        for (; done + EPQ <= len; done += EPQ) {
            T v[EPQ];
#pragma unroll
            for (int e = 0; e < EPQ; ++e) {
                srng::tinymt::step(s0, s1, s2, s3, p.x, p.y);
                v[e] = tconv<OUT>(srng::tinymt::temper(s0, s2, s3, p.z));
            }
            tst256(row + done, reinterpret_cast<const uint32_t *>(v));
        }
        for (; done < len; ++done) {
            srng::tinymt::step(s0, s1, s2, s3, p.x, p.y);
            row[done] = tconv<OUT>(srng::tinymt::temper(s0, s2, s3, p.z));
        }
        if (a.write_back) {
            a.state[s] = s0; a.state[ns + s] = s1; a.state[2 * ns + s] = s2; a.state[3 * ns + s] = s3;
        }
    }
}

unsigned grid_for(uint64_t count, uint64_t threads, uint64_t per_sm, const DeviceInfo &dev)
{
    uint64_t blocks = (count + threads - 1) / threads;
    const uint64_t cap = (uint64_t)dev.sm_count * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    return (unsigned)blocks;
}

}  // namespace

cudaError_t launch_tmt_place(uint32_t *state, uint64_t n_streams, const uint4 *params, uint64_t group_size,
                             const uint4 *seed_states, const uint4 *jt, int nbits, cudaStream_t stream,
                             const DeviceInfo &dev)
{
    k_tmt_place<<<grid_for(n_streams, kThreads, 8, dev), kThreads, 0, stream>>>(state, n_streams, params, group_size,
                                                                                 seed_states, jt, nbits);
    return cudaGetLastError();
}

cudaError_t launch_tmt_apply(uint32_t *state, uint64_t n_streams, const uint4 *params, uint64_t group_size,
                             uint64_t first, uint64_t count, const uint4 *poly, uint64_t g0, cudaStream_t stream,
                             const DeviceInfo &dev)
{
    if (count == 0) return cudaSuccess;
    k_tmt_apply<<<grid_for(count, kThreads, 8, dev), kThreads, 0, stream>>>(state, n_streams, params, group_size,
                                                                            first, count, poly, g0);
    return cudaGetLastError();
}

cudaError_t launch_tmt_generate(const TmtGenArgs &a, srng_out type, const srng_tune &t, cudaStream_t stream,
                                const DeviceInfo &dev)
{
    const uint64_t items = a.s_count * a.cps;
    const unsigned g = grid_for(items, kThreads, t.blocks_per_sm ? t.blocks_per_sm : 8, dev);
    switch (type) {
    case SRNG_OUT_U32: k_tmt_generate<SRNG_OUT_U32><<<g, kThreads, 0, stream>>>(a); break;
    case SRNG_OUT_F32: k_tmt_generate<SRNG_OUT_F32><<<g, kThreads, 0, stream>>>(a); break;
    case SRNG_OUT_EXP_F32: k_tmt_generate<SRNG_OUT_EXP_F32><<<g, kThreads, 0, stream>>>(a); break;
    case SRNG_OUT_NORMAL_F32: k_tmt_generate<SRNG_OUT_NORMAL_F32><<<g, kThreads, 0, stream>>>(a); break;
    default: k_tmt_generate<SRNG_OUT_F64><<<g, kThreads, 0, stream>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace srng_impl
