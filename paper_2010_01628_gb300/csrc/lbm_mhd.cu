// lbm_mhd.cu -- magnetohydrodynamic step (Sec. III.F of arXiv:2010.01628):
// the single-phase CM step driven by the Lorentz force F = j x b, coupled to
// vector-valued magnetic populations (per-node update in lbm_mhd.cuh).
#include "lbm_mhd.cuh"
#include "lbm_internal.h"
#include "lbm_reduce.cuh"

namespace lbm {

template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(256) mhd_step_kernel(const S* __restrict__ src, S* __restrict__ dst, MhdArgs p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.box.nx) return;
    mhd_node<S, C, WALLS, true>(src, dst, p, x, blockIdx.y, blockIdx.z);
}

template <typename S, typename C>
__global__ void mhd_init_kernel(S* __restrict__ dst, const double* __restrict__ slab, Box b, int z0, int nzs,
                                bool uniform) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, zs = blockIdx.z;
    if (x >= b.nx || zs >= nzs) return;
    const size_t m = (size_t)b.nx * b.ny * nzs;
    const size_t k = ((size_t)zs * b.ny + y) * b.nx + x;
    const uint32_t self = ((uint32_t)(z0 + zs) * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    C rho = (C)1, drho = (C)0, ux = (C)0, uy = (C)0, uz = (C)0;
    C bb[3] = {(C)0, (C)0, (C)0};
    if (!uniform) {
        drho = (C)(slab[k] - 1.0);
        rho = (C)slab[k];
        ux = (C)slab[m + k];
        uy = (C)slab[2 * m + k];
        uz = (C)slab[3 * m + k];
        bb[0] = (C)slab[5 * m + k];
        bb[1] = (C)slab[6 * m + k];
        bb[2] = (C)slab[7 * m + k];
    }
    C f[Q];
    equilibrium_shifted<C>(rho, drho, ux, uy, uz, f);
    scatter19<S, C>(dst, b.n, self, f);
    S* gdst = dst + (size_t)Q * b.n;
    store_geq<S, C, 0>(gdst, b.n, self, ux, uy, uz, bb);
    store_geq<S, C, 1>(gdst, b.n, self, ux, uy, uz, bb);
    store_geq<S, C, 2>(gdst, b.n, self, ux, uy, uz, bb);
    store_geq<S, C, 3>(gdst, b.n, self, ux, uy, uz, bb);
    store_geq<S, C, 4>(gdst, b.n, self, ux, uy, uz, bb);
    store_geq<S, C, 5>(gdst, b.n, self, ux, uy, uz, bb);
    store_geq<S, C, 6>(gdst, b.n, self, ux, uy, uz, bb);
}

template <typename S, typename C, bool WALLS>
__global__ void mhd_fields_kernel(const S* __restrict__ src, double* __restrict__ slab, MhdArgs p, int z0, int nzs) {
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
    gather19<S, C, WALLS>(src, b, q, x, y, z, self, (C)0, (C)0, (C)0, f);
    const C bw[3] = {(C)p.bw[0], (C)p.bw[1], (C)p.bw[2]};
    C g[7][3];
    gather_mag<S, C, WALLS>(src + (size_t)Q * b.n, b, q, x, y, z, self, bw, g);
    const Moments<C> mo = moments19(f);
    C bb[3];
    const Macro<C> a = mhd_macro<C>(mo, g, p, bb);
    slab[k] = (double)a.rho;
    slab[m + k] = (double)a.ux;
    slab[2 * m + k] = (double)a.uy;
    slab[3 * m + k] = (double)a.uz;
    slab[5 * m + k] = (double)bb[0];
    slab[6 * m + k] = (double)bb[1];
    slab[7 * m + k] = (double)bb[2];
}

template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(RED_THREADS) mhd_reduce_kernel(const S* __restrict__ src, MhdArgs p,
                                                                 C* __restrict__ uprev, bool have_prev, bool record,
                                                                 double* __restrict__ partials) {
    const Box& b = p.box;
    const int chunks_x = (b.nx + RED_THREADS - 1) / RED_THREADS;
    const long total = (long)chunks_x * b.ny * b.nz;
    RedAcc acc;
    acc.zero();
    const C bw[3] = {(C)p.bw[0], (C)p.bw[1], (C)p.bw[2]};
    for (long ch = blockIdx.x; ch < total; ch += gridDim.x) {
        const int cxk = (int)(ch % chunks_x);
        const long row = ch / chunks_x;
        const int y = (int)(row % b.ny), z = (int)(row / b.ny);
        const int x = cxk * RED_THREADS + threadIdx.x;
        if (x < b.nx) {
            const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
            const Nbr q = make_nbr(b, x, y, z);
            C f[Q];
            gather19<S, C, WALLS>(src, b, q, x, y, z, self, (C)0, (C)0, (C)0, f);
            C g[7][3];
            gather_mag<S, C, WALLS>(src + (size_t)Q * b.n, b, q, x, y, z, self, bw, g);
            const Moments<C> mo = moments19(f);
            C bb[3];
            const Macro<C> a = mhd_macro<C>(mo, g, p, bb);
            reduce_node<C>(acc, a.rho, a.ux, a.uy, a.uz, uprev, b.n, self, have_prev, record);
        }
    }
    block_reduce_store(acc, partials);
}

// ---------------------------------------------------------------------------
static MhdArgs mhd_args(const lbm_ctx* c) {
    MhdArgs p;
    p.box = c->box;
    p.omega = c->relax.omega;
    p.tau_m = c->phys.tau_m;
    p.inv_tau_m = 1.0 / c->phys.tau_m;
    p.jfac = 1.0 / (c->phys.tau_m * CSM2);
    for (int a = 0; a < 3; ++a) {
        p.g[a] = c->forcing.g[a];
        p.bw[a] = c->phys.b_wall[a];
    }
    return p;
}

template <typename S, typename C>
static cudaError_t step_t(lbm_ctx* c, long n, bool dry) {
    const MhdArgs p = mhd_args(c);
    const bool walls = (c->box.periodic & 7u) != 7u;
    const int bx = c->block_x;
    const dim3 grid = step_grid(c->box, bx);
    for (long s = 0; s < n; ++s) {
        const S* src = (const S*)c->buf[c->cur];
        S* dst = (S*)c->buf[c->cur ^ 1];
        if (walls)
            mhd_step_kernel<S, C, true><<<grid, bx, 0, c->stream>>>(src, dst, p);
        else
            mhd_step_kernel<S, C, false><<<grid, bx, 0, c->stream>>>(src, dst, p);
        if (!dry) c->cur ^= 1;
    }
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t init_t(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform) {
    const int bx = c->block_x;
    dim3 grid((unsigned)((c->box.nx + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)nzs);
    mhd_init_kernel<S, C><<<grid, bx, 0, c->stream>>>((S*)c->buf[c->cur], slab, c->box, z0, nzs, uniform);
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t fields_t(lbm_ctx* c, double* slab, int z0, int nzs) {
    const MhdArgs p = mhd_args(c);
    const int bx = c->block_x;
    dim3 grid((unsigned)((c->box.nx + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)nzs);
    if ((c->box.periodic & 7u) != 7u)
        mhd_fields_kernel<S, C, true><<<grid, bx, 0, c->stream>>>((const S*)c->buf[c->cur], slab, p, z0, nzs);
    else
        mhd_fields_kernel<S, C, false><<<grid, bx, 0, c->stream>>>((const S*)c->buf[c->cur], slab, p, z0, nzs);
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t reduce_t(lbm_ctx* c, bool record) {
    const MhdArgs p = mhd_args(c);
    if ((c->box.periodic & 7u) != 7u)
        mhd_reduce_kernel<S, C, true><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            (const S*)c->buf[c->cur], p, (C*)c->uprev, c->have_prev, record, c->partials);
    else
        mhd_reduce_kernel<S, C, false><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            (const S*)c->buf[c->cur], p, (C*)c->uprev, c->have_prev, record, c->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce_finalize(c);
}

cudaError_t mhd_step(lbm_ctx* c, long n, bool dry) {
    return c->prec == LBM_FP64 ? step_t<double, double>(c, n, dry) : step_t<float, float>(c, n, dry);
}
cudaError_t mhd_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform) {
    return c->prec == LBM_FP64 ? init_t<double, double>(c, slab, z0, nzs, uniform)
                               : init_t<float, float>(c, slab, z0, nzs, uniform);
}
cudaError_t mhd_fields(lbm_ctx* c, double* slab, int z0, int nzs) {
    return c->prec == LBM_FP64 ? fields_t<double, double>(c, slab, z0, nzs) : fields_t<float, float>(c, slab, z0, nzs);
}
cudaError_t mhd_reduce(lbm_ctx* c, bool record) {
    return c->prec == LBM_FP64 ? reduce_t<double, double>(c, record) : reduce_t<float, float>(c, record);
}

}  // namespace lbm
