// The CTA-wide status counters of the step kernels (one atomic per CTA and
// counter) and the tile constants they share.
#pragma once

#include <cuda_runtime.h>

#include "pab_bits.cuh"
#include "pab_check.cuh"
#include "pab_internal.h"

namespace pab {
namespace {

constexpr int kTile = 32;
constexpr int kMaxWarps = 16;

// Block-wide sums of the status counters, one atomic per CTA and counter.
__device__ __forceinline__ void flush_counters(uint32_t fl_or, uint32_t n_flag, uint32_t n_att,
                                               uint32_t n64, Counters *cnt)
{
    __shared__ uint32_t sc[4][kMaxWarps];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    fl_or = __reduce_or_sync(0xffffffffu, fl_or);
    n_flag = __reduce_add_sync(0xffffffffu, n_flag);
    n_att = __reduce_add_sync(0xffffffffu, n_att);
    n64 = __reduce_add_sync(0xffffffffu, n64);
    if (lane == 0) {
        sc[0][warp] = fl_or;
        sc[1][warp] = n_flag;
        sc[2][warp] = n_att;
        sc[3][warp] = n64;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t f = 0;
        unsigned long long a = 0, b = 0, d = 0;
        for (int w = 0; w < nw; ++w) {
            f |= sc[0][w];
            a += sc[1][w];
            b += sc[2][w];
            d += sc[3][w];
        }
        if (f)
            atomicOr(&cnt->flags_or, f);
        if (a)
            atomicAdd(&cnt->n_flagged, a);
        if (b)
            atomicAdd(&cnt->n_attempts, b);
        if (d)
            atomicAdd(&cnt->n_fp64, d);
    }
}

}  // namespace
}  // namespace pab
