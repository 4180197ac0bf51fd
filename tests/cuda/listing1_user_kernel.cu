// A user kernel written against include/srng_device.cuh, shaped like the
// paper's Listing 1 (Sec. 5): the host places the streams once (srng_create),
// each thread constructs its generator from the set's device view and calls
// next() -- here several times, writing its draws and storing the state back
// so a later launch continues the stream.  Built by the test with nvcc.
#include <cuda_runtime.h>
#include <stdint.h>

#include "srng.h"
#include "srng_device.cuh"

__global__ void listing1_mrg(float *ddata, srng_dev_view v, int per_thread)
{
    const uint64_t s = (uint64_t)blockDim.x * blockIdx.x + threadIdx.x;
    if (s >= v.n_streams) return;
    srng::Mrg32k3a rng(v, s);
    for (int k = 0; k < per_thread; ++k) ddata[s * per_thread + k] = rng.next_f32();
    rng.store(v, s);
}

__global__ void listing1_philox(uint32_t *ddata, srng_dev_view v, int per_thread)
{
    const uint64_t s = (uint64_t)blockDim.x * blockIdx.x + threadIdx.x;
    if (s >= v.n_streams) return;
    srng::Philox4x32_10 rng(v, s);
    for (int k = 0; k < per_thread; ++k) ddata[s * per_thread + k] = rng.next_u32();
    rng.store(v);
}

// Normal variates inside a user kernel: each thread draws FP32 uniform pairs
// from its own stream and turns them into Box-Muller pairs with srng::dist.
__global__ void user_normals(float *ddata, srng_dev_view v, int pairs)
{
    const uint64_t s = (uint64_t)blockDim.x * blockIdx.x + threadIdx.x;
    if (s >= v.n_streams) return;
    srng::Philox4x32_10 rng(v, s);
    for (int k = 0; k < pairs; ++k) {
        const float u0 = rng.next_f32(), u1 = rng.next_f32();
        srng::dist::normal_pair(u0, u1, &ddata[s * 2 * pairs + 2 * k], &ddata[s * 2 * pairs + 2 * k + 1]);
    }
    rng.store(v);
}

// Threefry stream handles in a user kernel (the same shape as listing1_philox).
__global__ void user_threefry(uint32_t *ddata, srng_dev_view v, int per_thread)
{
    const uint64_t s = (uint64_t)blockDim.x * blockIdx.x + threadIdx.x;
    if (s >= v.n_streams) return;
    srng::Threefry4x32_20 rng(v, s);
    for (int k = 0; k < per_thread; ++k) ddata[s * per_thread + k] = rng.next_u32();
    rng.store(v);
}

extern "C" int run_user_threefry(const srng_dev_view *v, uint32_t *out, int per_thread)
{
    const unsigned threads = 128, blocks = (unsigned)((v->n_streams + threads - 1) / threads);
    user_threefry<<<blocks, threads>>>(out, *v, per_thread);
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}

// The 64-bit-word Threefry form: one cipher block serves eight draws.
__global__ void user_threefry64(uint32_t *ddata, srng_dev_view v, int per_thread)
{
    const uint64_t s = (uint64_t)blockDim.x * blockIdx.x + threadIdx.x;
    if (s >= v.n_streams) return;
    srng::Threefry4x64_20 rng(v, s);
    for (int k = 0; k < per_thread; ++k) ddata[s * per_thread + k] = rng.next_u32();
    rng.store(v);
}

extern "C" int run_user_threefry64(const srng_dev_view *v, uint32_t *out, int per_thread)
{
    const unsigned threads = 128, blocks = (unsigned)((v->n_streams + threads - 1) / threads);
    user_threefry64<<<blocks, threads>>>(out, *v, per_thread);
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}

extern "C" int run_user_normals(const srng_dev_view *v, float *out, int pairs)
{
    const unsigned threads = 128, blocks = (unsigned)((v->n_streams + threads - 1) / threads);
    user_normals<<<blocks, threads>>>(out, *v, pairs);
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}

extern "C" int run_listing1(const srng_dev_view *v, void *out, int per_thread)
{
    const unsigned threads = 128, blocks = (unsigned)((v->n_streams + threads - 1) / threads);
    if (v->gen == SRNG_MRG32K3A) listing1_mrg<<<blocks, threads>>>((float *)out, *v, per_thread);
    else listing1_philox<<<blocks, threads>>>((uint32_t *)out, *v, per_thread);
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}

// next4(): four draws per call, `quads` calls per thread, the state stored back.
template <class Gen>
__global__ void user_next4(uint4 *ddata, srng_dev_view v, int quads)
{
    const uint64_t s = (uint64_t)blockDim.x * blockIdx.x + threadIdx.x;
    if (s >= v.n_streams) return;
    Gen rng(v, s);
    for (int k = 0; k < quads; ++k) ddata[s * quads + k] = rng.next4();
    if constexpr (std::is_same<Gen, srng::Mrg32k3a>::value || std::is_same<Gen, srng::TinyMT32>::value)
        rng.store(v, s);
    else
        rng.store(v);
}

extern "C" int run_user_next4(const srng_dev_view *v, uint4 *out, int quads)
{
    const unsigned threads = 128, blocks = (unsigned)((v->n_streams + threads - 1) / threads);
    switch (v->gen) {
    case SRNG_MRG32K3A: user_next4<srng::Mrg32k3a><<<blocks, threads>>>(out, *v, quads); break;
    case SRNG_THREEFRY4X32_20: user_next4<srng::Threefry4x32_20><<<blocks, threads>>>(out, *v, quads); break;
    case SRNG_THREEFRY4X64_20: user_next4<srng::Threefry4x64_20><<<blocks, threads>>>(out, *v, quads); break;
    case SRNG_TINYMT32: user_next4<srng::TinyMT32><<<blocks, threads>>>(out, *v, quads); break;
    default: user_next4<srng::Philox4x32_10><<<blocks, threads>>>(out, *v, quads); break;
    }
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}

// Stream handles built at an offset: thread s reads `per` draws starting
// offsets[s] draws after stream s's position (MRG32k3a by jump-ahead on the
// device, the counter-based ones by moving the position).
template <class Gen>
__global__ void user_offset(uint32_t *ddata, srng_dev_view v, const uint64_t *offsets, int per)
{
    const uint64_t s = (uint64_t)blockDim.x * blockIdx.x + threadIdx.x;
    if (s >= v.n_streams) return;
    Gen rng(v, s, offsets[s]);
    for (int k = 0; k < per; ++k) ddata[s * per + k] = rng.next_u32();
}

extern "C" int run_user_offset(const srng_dev_view *v, uint32_t *out, const uint64_t *offsets, int per)
{
    const unsigned threads = 128, blocks = (unsigned)((v->n_streams + threads - 1) / threads);
    switch (v->gen) {
    case SRNG_MRG32K3A: user_offset<srng::Mrg32k3a><<<blocks, threads>>>(out, *v, offsets, per); break;
    case SRNG_THREEFRY4X32_20: user_offset<srng::Threefry4x32_20><<<blocks, threads>>>(out, *v, offsets, per); break;
    case SRNG_THREEFRY4X64_20: user_offset<srng::Threefry4x64_20><<<blocks, threads>>>(out, *v, offsets, per); break;
    default: user_offset<srng::Philox4x32_10><<<blocks, threads>>>(out, *v, offsets, per); break;
    }
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}
