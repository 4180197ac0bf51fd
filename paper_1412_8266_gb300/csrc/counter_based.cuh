// Counter-based block functions of the library's kernels (paper Sec. 4.3):
// one entry point for Philox4x32-10, Threefry4x32-20 and Threefry4x64-20 so
// the generation and batch kernels are written once for all three.
//
// The kernels work in 4-word blocks: block q of a stream holds draws 4q..4q+3.
// Philox: counter (q, c2, c3), key (kk0, kk1).  Threefry4x32: counter (q, 0, 0),
// key (kk0, kk1, c2, c3).  Threefry4x64: one 64-bit block Q gives eight words,
// so 4-word block q is half q mod 2 of block Q = q / 2 under the 64-bit key
// (kk1:kk0, c3:c2, 0, 0).  The callers fill (kk0, kk1, c2, c3) from the set:
// counter-split Philox (seed, stream), keyed Philox (stream, seed), Threefry
// (stream, seed).
#pragma once
#include <stdint.h>

#include "srng_device.cuh"

namespace srng_impl {

enum { kCipherPhilox = 0, kCipherThreefry = 1, kCipherThreefry64 = 2 };

// The generation kernels start a stream's run at the cipher block that holds
// its position: words per block minus one is the largest offset of the first
// draw inside that block (3 for the 4-word blocks, 7 for Threefry4x64).
template <int CIPHER> __host__ __device__ constexpr uint32_t cb_align_mask() { return CIPHER == kCipherThreefry64 ? 7u : 3u; }

// 4-word block q (x0, x1 = q on entry).
template <int CIPHER>
__device__ __forceinline__ void cb_block(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3, uint32_t kk0,
                                         uint32_t kk1, uint32_t c2, uint32_t c3)
{
    if constexpr (CIPHER == kCipherPhilox) {
        x2 = c2;
        x3 = c3;
        srng::philox::block(x0, x1, x2, x3, kk0, kk1);
    } else if constexpr (CIPHER == kCipherThreefry) {
        x2 = 0;
        x3 = 0;
        srng::threefry::block(x0, x1, x2, x3, kk0, kk1, c2, c3);
    } else {
        const uint64_t q = (uint64_t)x1 << 32 | x0;
        uint32_t w[8];
        srng::threefry64::words(q >> 1, (uint64_t)kk1 << 32 | kk0, (uint64_t)c3 << 32 | c2, w);
        const bool hi = q & 1;
        x0 = hi ? w[4] : w[0];
        x1 = hi ? w[5] : w[1];
        x2 = hi ? w[6] : w[2];
        x3 = hi ? w[7] : w[3];
    }
}

// 4-word blocks q and q + 1 into w[0..7].  For Threefry4x64 an even q is one
// 64-bit block (computed once); an odd q straddles two.  EVEN: the caller
// guarantees an even q (no code for the straddling case).
template <int CIPHER, bool EVEN = false>
__device__ __forceinline__ void cb_pair(uint64_t q, uint32_t *w, uint32_t kk0, uint32_t kk1, uint32_t c2, uint32_t c3)
{
    if constexpr (CIPHER == kCipherThreefry64) {
        if (EVEN || (q & 1) == 0) {
            srng::threefry64::words(q >> 1, (uint64_t)kk1 << 32 | kk0, (uint64_t)c3 << 32 | c2, w);
            return;
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint64_t qh = q + h;
        w[4 * h] = (uint32_t)qh;
        w[4 * h + 1] = (uint32_t)(qh >> 32);
        cb_block<CIPHER>(w[4 * h], w[4 * h + 1], w[4 * h + 2], w[4 * h + 3], kk0, kk1, c2, c3);
    }
}

}  // namespace srng_impl
