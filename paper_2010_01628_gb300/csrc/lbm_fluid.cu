// lbm_fluid.cu -- single-phase D3Q19 central-moment step (Sec. II of
// arXiv:2010.01628) with a constant body force, in four storage precisions.
//
// One thread per node, a block along x.  Each step is one fused pass:
// pull the 19 post-collision populations of the neighbours (periodic wrap or
// half-way bounce-back), form rho and u = (sum f c + F/2)/rho, relax the five
// deviatoric central second moments by (1 - omega), set every other central
// moment to its forced equilibrium value, rebuild f* with the two-step
// transform of App. C and store it, coalesced, to the other buffer.
#include "lbm_fluid.cuh"
#include "lbm_internal.h"
#include "lbm_reduce.cuh"

namespace lbm {

template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(256) fluid_step_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                         FluidArgs p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.box.nx) return;
    fluid_node<S, C, WALLS, true>(src, dst, p, x, blockIdx.y, blockIdx.z);
}

// Equilibrium initialisation of a z-slab from FP64 fields (rho, ux, uy, uz
// planes of nx*ny*nzs values), or of the uniform rest state.
template <typename S, typename C>
__global__ void fluid_init_kernel(S* __restrict__ dst, const double* __restrict__ slab, Box b, int z0, int nzs,
                                  bool uniform) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, zs = blockIdx.z;
    if (x >= b.nx || zs >= nzs) return;
    const size_t m = (size_t)b.nx * b.ny * nzs;
    const size_t k = ((size_t)zs * b.ny + y) * b.nx + x;
    const uint32_t self = ((uint32_t)(z0 + zs) * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    C rho = (C)1, drho = (C)0, ux = (C)0, uy = (C)0, uz = (C)0;
    if (!uniform) {
        drho = (C)(slab[k] - 1.0);  // the shift is taken in FP64
        rho = (C)slab[k];
        ux = (C)slab[m + k];
        uy = (C)slab[2 * m + k];
        uz = (C)slab[3 * m + k];
    }
    C f[Q];
    equilibrium_shifted<C>(rho, drho, ux, uy, uz, f);
    scatter19<S, C>(dst, b.n, self, f);
}

// Moments of the gathered state for a z-slab: rho, u (with +F/2).
template <typename S, typename C, bool WALLS>
__global__ void fluid_fields_kernel(const S* __restrict__ src, double* __restrict__ slab, FluidArgs p, int z0,
                                    int nzs) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, zs = blockIdx.z;
    const Box& b = p.box;
    if (x >= b.nx || zs >= nzs) return;
    const int z = z0 + zs;
    const size_t m = (size_t)b.nx * b.ny * nzs;
    const size_t k = ((size_t)zs * b.ny + y) * b.nx + x;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q];
    gather19<S, C, WALLS>(src, b, q, x, y, z, self, (C)p.lid[0], (C)p.lid[1], (C)p.lid[2], f);
    const Moments<C> mo = moments19(f);
    const Macro<C> a = fluid_macro(mo, (C)p.g[0], (C)p.g[1], (C)p.g[2]);
    slab[k] = (double)a.rho;
    slab[m + k] = (double)a.ux;
    slab[2 * m + k] = (double)a.uy;
    slab[3 * m + k] = (double)a.uz;
}

template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(RED_THREADS) fluid_reduce_kernel(const S* __restrict__ src, FluidArgs p,
                                                                   C* __restrict__ uprev, bool have_prev,
                                                                   bool record, double* __restrict__ partials) {
    const Box& b = p.box;
    const int chunks_x = (b.nx + RED_THREADS - 1) / RED_THREADS;
    const long total = (long)chunks_x * b.ny * b.nz;
    RedAcc acc;
    acc.zero();
    for (long ch = blockIdx.x; ch < total; ch += gridDim.x) {
        const int cxk = (int)(ch % chunks_x);
        const long row = ch / chunks_x;
        const int y = (int)(row % b.ny), z = (int)(row / b.ny);
        const int x = cxk * RED_THREADS + threadIdx.x;
        if (x < b.nx) {
            const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
            const Nbr q = make_nbr(b, x, y, z);
            C f[Q];
            gather19<S, C, WALLS>(src, b, q, x, y, z, self, (C)p.lid[0], (C)p.lid[1], (C)p.lid[2], f);
            const Moments<C> mo = moments19(f);
            const Macro<C> a = fluid_macro(mo, (C)p.g[0], (C)p.g[1], (C)p.g[2]);
            reduce_node<C>(acc, a.rho, a.ux, a.uy, a.uz, uprev, b.n, self, have_prev, record);
        }
    }
    block_reduce_store(acc, partials);
}

// ---------------------------------------------------------------------------
static FluidArgs fluid_args(const lbm_ctx* c) {
    FluidArgs p;
    p.box = c->box;
    p.omega = c->relax.omega;
    for (int a = 0; a < 3; ++a) {
        p.g[a] = c->forcing.g[a];
        p.lid[a] = (c->box.periodic & 2u) ? 0.0 : c->grid.lid_u[a];
    }
    return p;
}

template <typename S, typename C>
static cudaError_t step_t(lbm_ctx* c, long n, bool dry) {
    const FluidArgs p = fluid_args(c);
    const bool walls = (c->box.periodic & 7u) != 7u;
    const int bx = c->block_x;
    const dim3 grid = step_grid(c->box, bx);
    for (long s = 0; s < n; ++s) {
        const S* src = (const S*)c->buf[c->cur];
        S* dst = (S*)c->buf[c->cur ^ 1];
        if (walls)
            fluid_step_kernel<S, C, true><<<grid, bx, 0, c->stream>>>(src, dst, p);
        else
            fluid_step_kernel<S, C, false><<<grid, bx, 0, c->stream>>>(src, dst, p);
        if (!dry) c->cur ^= 1;
    }
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t init_t(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform) {
    const int bx = c->block_x;
    dim3 grid((unsigned)((c->box.nx + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)nzs);
    fluid_init_kernel<S, C><<<grid, bx, 0, c->stream>>>((S*)c->buf[c->cur], slab, c->box, z0, nzs, uniform);
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t fields_t(lbm_ctx* c, double* slab, int z0, int nzs) {
    const FluidArgs p = fluid_args(c);
    const int bx = c->block_x;
    dim3 grid((unsigned)((c->box.nx + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)nzs);
    if ((c->box.periodic & 7u) != 7u)
        fluid_fields_kernel<S, C, true><<<grid, bx, 0, c->stream>>>((const S*)c->buf[c->cur], slab, p, z0, nzs);
    else
        fluid_fields_kernel<S, C, false><<<grid, bx, 0, c->stream>>>((const S*)c->buf[c->cur], slab, p, z0, nzs);
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t reduce_t(lbm_ctx* c, bool record) {
    const FluidArgs p = fluid_args(c);
    if ((c->box.periodic & 7u) != 7u)
        fluid_reduce_kernel<S, C, true><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            (const S*)c->buf[c->cur], p, (C*)c->uprev, c->have_prev, record, c->partials);
    else
        fluid_reduce_kernel<S, C, false><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            (const S*)c->buf[c->cur], p, (C*)c->uprev, c->have_prev, record, c->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce_finalize(c);
}

cudaError_t fluid_step(lbm_ctx* c, long n, bool dry) {
    switch (c->prec) {
        case LBM_FP64: return step_t<double, double>(c, n, dry);
        case LBM_FP32: return step_t<float, float>(c, n, dry);
        case LBM_FP16_SHIFTED: return step_t<__half, float>(c, n, dry);
        case LBM_BF16_SHIFTED: return step_t<__nv_bfloat16, float>(c, n, dry);
    }
    return cudaErrorInvalidValue;
}
cudaError_t fluid_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform) {
    switch (c->prec) {
        case LBM_FP64: return init_t<double, double>(c, slab, z0, nzs, uniform);
        case LBM_FP32: return init_t<float, float>(c, slab, z0, nzs, uniform);
        case LBM_FP16_SHIFTED: return init_t<__half, float>(c, slab, z0, nzs, uniform);
        case LBM_BF16_SHIFTED: return init_t<__nv_bfloat16, float>(c, slab, z0, nzs, uniform);
    }
    return cudaErrorInvalidValue;
}
cudaError_t fluid_fields(lbm_ctx* c, double* slab, int z0, int nzs) {
    switch (c->prec) {
        case LBM_FP64: return fields_t<double, double>(c, slab, z0, nzs);
        case LBM_FP32: return fields_t<float, float>(c, slab, z0, nzs);
        case LBM_FP16_SHIFTED: return fields_t<__half, float>(c, slab, z0, nzs);
        case LBM_BF16_SHIFTED: return fields_t<__nv_bfloat16, float>(c, slab, z0, nzs);
    }
    return cudaErrorInvalidValue;
}
cudaError_t fluid_reduce(lbm_ctx* c, bool record) {
    switch (c->prec) {
        case LBM_FP64: return reduce_t<double, double>(c, record);
        case LBM_FP32: return reduce_t<float, float>(c, record);
        case LBM_FP16_SHIFTED: return reduce_t<__half, float>(c, record);
        case LBM_BF16_SHIFTED: return reduce_t<__nv_bfloat16, float>(c, record);
    }
    return cudaErrorInvalidValue;
}

// Deterministic final sum of the per-block partials (one block).
__global__ void reduce_finalize_kernel(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    __shared__ double sh[RED_THREADS][RED_WIDTH];
    double acc[RED_WIDTH];
#pragma unroll
    for (int k = 0; k < RED_WIDTH; ++k) acc[k] = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < RED_WIDTH; ++k) acc[k] += partials[(size_t)i * RED_WIDTH + k];
#pragma unroll
    for (int k = 0; k < RED_WIDTH; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < RED_WIDTH; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x < RED_WIDTH) out[threadIdx.x] = sh[0][threadIdx.x];
}

cudaError_t reduce_finalize(lbm_ctx* c) {
    reduce_finalize_kernel<<<1, RED_THREADS, 0, c->stream>>>(c->partials, RED_BLOCKS, c->result);
    return cudaGetLastError();
}

}  // namespace lbm
