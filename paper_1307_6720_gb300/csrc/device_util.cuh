// Small device helpers shared by the kernel translation units.
#pragma once

#include "mhs_internal.h"

namespace mhs {

__device__ __forceinline__ size_t at(const Geom& g, int i, int j, int k) {
    return size_t(i) + size_t(g.px) * (size_t(j) + size_t(g.ny) * size_t(k));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum in a fixed order (warp butterflies, then warp 0 over the
// per-warp sums); every thread of the block must call it.  The result is
// valid in every thread of warp 0, in particular thread 0.
template <typename T>
__device__ T block_sum(T v) {
    __shared__ T ws[32];
    const int lane = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    v = warp_sum(v);
    if ((lane & 31) == 0) ws[lane >> 5] = v;
    __syncthreads();
    T s = T(0);
    if (lane < 32) {
        s = (lane < (nthreads + 31) / 32) ? ws[lane] : T(0);
        s = warp_sum(s);
    }
    __syncthreads();
    return s;
}

}  // namespace mhs
