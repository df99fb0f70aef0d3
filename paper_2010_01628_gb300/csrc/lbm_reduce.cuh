// lbm_reduce.cuh -- FP64 block reduction used by the per-physics reduction
// kernels (mass, momentum, residual norms and a bad-node count).
#pragma once

#include "lbm_internal.h"

namespace lbm {

// Accumulator of one thread; reduced across the block with warp shuffles and
// written as one partial per block (no atomics: the result is deterministic).
struct RedAcc {
    double v[RED_WIDTH];
    __device__ void zero() {
#pragma unroll
        for (int k = 0; k < RED_WIDTH; ++k) v[k] = 0.0;
    }
};

__device__ __forceinline__ void block_reduce_store(RedAcc& a, double* __restrict__ partials) {
    __shared__ double sh[RED_THREADS / 32][RED_WIDTH];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < RED_WIDTH; ++k) {
        double x = a.v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < RED_WIDTH) {
        double s = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) s += sh[w][threadIdx.x];
        partials[(size_t)blockIdx.x * RED_WIDTH + threadIdx.x] = s;
    }
}

// Accumulate one node.  u_prev may be null (first reduction).  Records u.
template <typename C>
__device__ __forceinline__ void reduce_node(RedAcc& a, C rho, C ux, C uy, C uz, C* __restrict__ uprev, size_t n,
                                            uint32_t cell, bool have_prev, bool record) {
    const bool bad = !(rho > (C)0) || !isfinite((double)rho) || !isfinite((double)ux) || !isfinite((double)uy) ||
                     !isfinite((double)uz);
    if (bad) {
        a.v[6] += 1.0;
        return;
    }
    const double r = (double)rho, x = (double)ux, y = (double)uy, z = (double)uz;
    a.v[0] += r;
    a.v[1] += r * x;
    a.v[2] += r * y;
    a.v[3] += r * z;
    a.v[5] += x * x + y * y + z * z;
    if (have_prev) {
        const double dx = x - (double)uprev[cell], dy = y - (double)uprev[n + cell], dz = z - (double)uprev[2 * n + cell];
        a.v[4] += dx * dx + dy * dy + dz * dz;
    }
    if (record) {
        uprev[cell] = ux;
        uprev[n + cell] = uy;
        uprev[2 * n + cell] = uz;
    }
}

}  // namespace lbm
