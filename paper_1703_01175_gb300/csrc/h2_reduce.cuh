// Deterministic reductions shared by the Krylov kernels: warp and block sums
// of complex FP64 values, and the "last block to finish" test that lets one
// kernel combine the per-block partial sums of a grid in a fixed order.
#pragma once

#include <cuda_runtime.h>

namespace h2 {

static __device__ __forceinline__ double2 zsum2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

static __device__ __forceinline__ double2 warp_sum2(double2 v)
{
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// block-wide sum over NT threads (all threads get the result)
template <int NT>
static __device__ double2 block_sum2(double2 v)
{
    __shared__ double2 red[NT / 32];
    __shared__ double2 tot;
    v = warp_sum2(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 s = red[0];
        for (int q = 1; q < NT / 32; ++q) s = zsum2(s, red[q]);
        tot = s;
    }
    __syncthreads();
    return tot;
}

// true in the last block of the grid's x dimension to pass this point; the
// counter is reset for the next use. Partial sums written before the call by
// any block are visible to the last one.
static __device__ bool last_block(unsigned *ticket)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        last = atomicAdd(ticket, 1u) == (unsigned)gridDim.x - 1;
        if (last) *ticket = 0u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

}  // namespace h2
