// The paper's Listing 1 (Sec. 5), written against include/srng_device.cuh:
// the kernel constructs RNG<float, MRG32k3a> with no arguments and stores
// rng.next() at its global thread index; the host calls init before the
// launch and release after.  Built by the test with nvcc -std=c++20.
#include <cuda_runtime.h>
#include <stdint.h>

#include "srng.h"
#include "srng_device.cuh"

using srng::RNG;

__global__ void fooKernel(float *ddata)
{
    RNG<float, srng::Mrg32k3a> rng;
    ddata[blockDim.x * blockIdx.x + threadIdx.x] = rng.next();
}

__global__ void barKernel(uint32_t *ddata)
{
    RNG<uint32_t, srng::Philox4x32_10> rng;
    const uint64_t i = (uint64_t)blockDim.x * blockIdx.x + threadIdx.x;
    ddata[2 * i] = rng.next();
    ddata[2 * i + 1] = rng.next();
}

__global__ void bazKernel(double *ddata)
{
    RNG<double, srng::Threefry4x32_20> rng;
    ddata[blockDim.x * blockIdx.x + threadIdx.x] = rng.next();
}

__global__ void bazKernel64(double *ddata)
{
    RNG<double, srng::Threefry4x64_20> rng;
    ddata[blockDim.x * blockIdx.x + threadIdx.x] = rng.next();
}

__global__ void quxKernel(float *ddata)
{
    RNG<float, srng::TinyMT32> rng;   // the block's threads share one parameter set
    const uint64_t i = (uint64_t)blockDim.x * blockIdx.x + threadIdx.x;
    ddata[2 * i] = rng.next();
    ddata[2 * i + 1] = rng.next();
}

// launches = number of fooKernel launches (each continues every stream).
extern "C" int run_paper_listing1(float *d_data, int block_num, int thread_num, int launches, uint64_t seed)
{
    if (RNG<float, srng::Mrg32k3a>::init((uint64_t)block_num * thread_num, seed) != SRNG_OK) return 1;
    for (int l = 0; l < launches; ++l)
        fooKernel<<<block_num, thread_num>>>(d_data + (size_t)l * block_num * thread_num);
    const int rc = cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
    RNG<float, srng::Mrg32k3a>::release();
    return rc;
}

extern "C" int run_philox_form(uint32_t *d_data, int block_num, int thread_num, uint64_t seed)
{
    if (RNG<uint32_t, srng::Philox4x32_10>::init((uint64_t)block_num * thread_num, seed) != SRNG_OK) return 1;
    barKernel<<<block_num, thread_num>>>(d_data);
    const int rc = cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
    RNG<uint32_t, srng::Philox4x32_10>::release();
    return rc;
}

extern "C" int run_threefry_form(double *d_data, int block_num, int thread_num, uint64_t seed)
{
    if (RNG<double, srng::Threefry4x32_20>::init((uint64_t)block_num * thread_num, seed) != SRNG_OK) return 1;
    bazKernel<<<block_num, thread_num>>>(d_data);
    const int rc = cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
    RNG<double, srng::Threefry4x32_20>::release();
    return rc;
}

extern "C" int run_threefry64_form(double *d_data, int block_num, int thread_num, uint64_t seed)
{
    if (RNG<double, srng::Threefry4x64_20>::init((uint64_t)block_num * thread_num, seed) != SRNG_OK) return 1;
    bazKernel64<<<block_num, thread_num>>>(d_data);
    const int rc = cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
    RNG<double, srng::Threefry4x64_20>::release();
    return rc;
}

extern "C" int run_tinymt_form(float *d_data, int block_num, int thread_num, uint64_t seed)
{
    if (RNG<float, srng::TinyMT32>::init((uint64_t)block_num * thread_num, seed) != SRNG_OK) return 1;
    quxKernel<<<block_num, thread_num>>>(d_data);
    const int rc = cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
    RNG<float, srng::TinyMT32>::release();
    return rc;
}
