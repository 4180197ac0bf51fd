// Every form of the MRG32k3a double in the device header against the
// integer-built one, for every z in [1, m1]: the generation kernels mix them
// (a share of each row through the FP64 unit), so they must agree bit for bit.
// The integer-built form itself is compared with the IEEE product elsewhere.
#include <stdint.h>

#include "srng_device.cuh"

namespace {

__global__ void k_forms(uint64_t z0, uint64_t n, unsigned long long *bad, unsigned long long *first)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t z = (uint32_t)(z0 + i);
        const long long a = __double_as_longlong(srng::mrg::to_f64(z));
        const long long b = __double_as_longlong(srng::mrg::to_f64_dmul(z));
        const long long c = __double_as_longlong(srng::mrg::to_f64_fma(z));
        if (a != b || a != c) {
            atomicAdd(bad, 1ull);
            atomicMin(first, (unsigned long long)z);
        }
    }
}

}  // namespace

// Checks z in [z0, z0 + n); returns 0 and the number of disagreeing z (and
// the smallest such z) through the two host pointers, or a CUDA error code.
extern "C" int run_mrg_f64_forms(uint64_t z0, uint64_t n, unsigned long long *bad_out,
                                 unsigned long long *first_out)
{
    unsigned long long *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) return (int)e;
    const unsigned long long init[2] = {0ull, ~0ull};
    e = cudaMemcpy(d, init, sizeof init, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_forms<<<1216, 256>>>(z0, n, d, d + 1);
        e = cudaGetLastError();
    }
    unsigned long long h[2] = {0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    *bad_out = h[0];
    *first_out = h[1];
    return (int)e;
}
