// K1 -- stream placement and jump-ahead on the device (paper Sec. 2.3 sequence
// splitting, Sec. 4.1 MRG32k3a streams of 2^127 and substreams of 2^76).
//
// Placement: stream i of a set starts at B^i y0, B = A^(2^e).  With
// J_k = B^(2^k) prepared on the host, one thread per stream multiplies y0 by
// J_k for every set bit k of i: at most 64 exact 3x3 modular matrix-vector
// products per component, no sequential dependence between streams.
//
// HBM traffic per stream: 24 bytes written (placement), 24 read + 24 written
// (apply).  Both are small next to generation and are launched with a grid of
// at most 8 blocks of 256 threads per SM.
#include "internal.h"
#include "srng_device.cuh"

namespace srng_impl {

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
    k_mrg_place(uint32_t *__restrict__ st, uint64_t ns, uint64_t first, uint64_t count, uint64_t index_base,
                uint32_t y0, uint32_t y1, uint32_t y2, uint32_t y3, uint32_t y4, uint32_t y5,
                const __grid_constant__ JumpTable tab, int nbits)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const uint64_t slot = first + i;          // storage slot in the set
        const uint64_t idx = index_base + slot;   // stream number in the whole sequence
        uint32_t s0 = y0, s1 = y1, s2 = y2, s3 = y3, s4 = y4, s5 = y5;
        for (int k = 0; k < nbits; ++k)
            if ((idx >> k) & 1) srng::mrg::jump(tab.m[k], s0, s1, s2, s3, s4, s5);
        st[0 * ns + slot] = s0; st[1 * ns + slot] = s1; st[2 * ns + slot] = s2;
        st[3 * ns + slot] = s3; st[4 * ns + slot] = s4; st[5 * ns + slot] = s5;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_mrg_apply(uint32_t *__restrict__ st, uint64_t ns, uint64_t first, uint64_t count, const MatPair m)
{
    // launched as a programmatic dependent of a generation kernel: wait until
    // that kernel has finished reading the states (no-op otherwise)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const uint64_t idx = first + i;
        uint32_t s0 = st[0 * ns + idx], s1 = st[1 * ns + idx], s2 = st[2 * ns + idx];
        uint32_t s3 = st[3 * ns + idx], s4 = st[4 * ns + idx], s5 = st[5 * ns + idx];
        srng::mrg::jump(m.a, s0, s1, s2, s3, s4, s5);
        st[0 * ns + idx] = s0; st[1 * ns + idx] = s1; st[2 * ns + idx] = s2;
        st[3 * ns + idx] = s3; st[4 * ns + idx] = s4; st[5 * ns + idx] = s5;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_philox_advance(uint64_t *__restrict__ pos, uint64_t first, uint64_t count, uint64_t n)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        pos[first + i] += n;
}

unsigned grid_for(uint64_t count, const DeviceInfo &dev)
{
    uint64_t blocks = (count + kThreads - 1) / kThreads;
    uint64_t cap = (uint64_t)dev.sm_count * 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    return (unsigned)blocks;
}

}  // namespace

cudaError_t launch_mrg_place(uint32_t *state, uint64_t n_streams, uint64_t first, uint64_t count,
                             uint64_t index_base, const uint32_t y0[6], const JumpTable &tab, int nbits,
                             cudaStream_t stream, const DeviceInfo &dev)
{
    if (count == 0) return cudaSuccess;
    k_mrg_place<<<grid_for(count, dev), kThreads, 0, stream>>>(state, n_streams, first, count, index_base, y0[0],
                                                               y0[1], y0[2], y0[3], y0[4], y0[5], tab, nbits);
    return cudaGetLastError();
}

cudaError_t launch_mrg_apply(uint32_t *state, uint64_t n_streams, uint64_t first, uint64_t count,
                             const MatPair &m, cudaStream_t stream, const DeviceInfo &dev, bool dependent)
{
    if (count == 0) return cudaSuccess;
    if (!dependent) {
        k_mrg_apply<<<grid_for(count, dev), kThreads, 0, stream>>>(state, n_streams, first, count, m);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid_for(count, dev));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mrg_apply, state, n_streams, first, count, m);
}

cudaError_t launch_philox_advance(uint64_t *pos, uint64_t first, uint64_t count, uint64_t n,
                                  cudaStream_t stream, const DeviceInfo &dev)
{
    if (count == 0 || n == 0) return cudaSuccess;
    k_philox_advance<<<grid_for(count, dev), kThreads, 0, stream>>>(pos, first, count, n);
    return cudaGetLastError();
}

}  // namespace srng_impl
