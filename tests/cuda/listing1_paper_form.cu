// Device-header usage in the form the paper's Listing 1 describes (Sec. 5):
// a kernel builds srng::RNG<T, Gen> with no arguments, so the object takes
// the stream of its global thread index from the set that the static host
// init() bound before the launch, and release() frees that set afterwards.
// One templated kernel and one host driver serve every generator; built by
// the test with nvcc -std=c++20 (so the C++20 concept check is compiled too).
#include <cuda_runtime.h>
#include <stdint.h>

#include "srng.h"
#include "srng_device.cuh"

// K draws per thread, thread t's draws at out[K t .. K t + K - 1].
template <class T, class Gen, int K>
__global__ void draws_per_thread(T *out)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    srng::RNG<T, Gen> gen;  // the stream of thread t; its state is stored back when gen goes out of scope
#pragma unroll
    for (int k = 0; k < K; ++k) out[K * t + k] = gen.next();
}

// init for blocks x threads streams, `launches` launches (each continues every
// stream; launch l writes at out + l * blocks * threads * K), release.
template <class T, class Gen, int K>
static int drive(T *out, int blocks, int threads, uint64_t seed, int launches)
{
    const uint64_t n = (uint64_t)blocks * threads;
    if (srng::RNG<T, Gen>::init(n, seed) != SRNG_OK) return 1;
    for (int l = 0; l < launches; ++l) draws_per_thread<T, Gen, K><<<blocks, threads>>>(out + (size_t)l * n * K);
    const int rc = cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
    srng::RNG<T, Gen>::release();
    return rc;
}

extern "C" int run_listing1_form(float *out, int blocks, int threads, int launches, uint64_t seed)
{
    return drive<float, srng::Mrg32k3a, 1>(out, blocks, threads, seed, launches);
}

extern "C" int run_philox_form(uint32_t *out, int blocks, int threads, uint64_t seed)
{
    return drive<uint32_t, srng::Philox4x32_10, 2>(out, blocks, threads, seed, 1);
}

extern "C" int run_threefry_form(double *out, int blocks, int threads, uint64_t seed)
{
    return drive<double, srng::Threefry4x32_20, 1>(out, blocks, threads, seed, 1);
}

extern "C" int run_threefry64_form(double *out, int blocks, int threads, uint64_t seed)
{
    return drive<double, srng::Threefry4x64_20, 1>(out, blocks, threads, seed, 1);
}

// TinyMT32: the threads of a 256-thread block share one parameter set.
extern "C" int run_tinymt_form(float *out, int blocks, int threads, uint64_t seed)
{
    return drive<float, srng::TinyMT32, 2>(out, blocks, threads, seed, 1);
}
