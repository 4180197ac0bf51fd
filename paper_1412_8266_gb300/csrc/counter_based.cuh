// Counter-based block functions of the library's kernels (paper Sec. 4.3):
// one entry point for Philox4x32-10 and Threefry4x32-20 so the generation and
// batch kernels are written once for both.
//
// On entry x0, x1 hold the block index q (low, high).  Philox: counter words
// 2-3 = (c2, c3), key = (kk0, kk1).  Threefry: counter words 2-3 = 0,
// key = (kk0, kk1, c2, c3).  The callers fill (kk0, kk1, c2, c3) from the set:
// counter-split Philox (seed, stream), keyed Philox (stream, seed), Threefry
// (stream, seed).
#pragma once
#include <stdint.h>

#include "srng_device.cuh"

namespace srng_impl {

enum { kCipherPhilox = 0, kCipherThreefry = 1 };

template <int CIPHER>
__device__ __forceinline__ void cb_block(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3, uint32_t kk0,
                                         uint32_t kk1, uint32_t c2, uint32_t c3)
{
    if constexpr (CIPHER == kCipherPhilox) {
        x2 = c2;
        x3 = c3;
        srng::philox::block(x0, x1, x2, x3, kk0, kk1);
    } else {
        x2 = 0;
        x3 = 0;
        srng::threefry::block(x0, x1, x2, x3, kk0, kk1, c2, c3);
    }
}

}  // namespace srng_impl
