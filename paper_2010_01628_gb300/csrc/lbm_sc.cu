// lbm_sc.cu -- Shan-Chen pseudopotential multiphase step (Sec. III.G of
// arXiv:2010.01628, the static-bubble test).
//
// Two passes per step, both pulling the single-phase population set.  Pass 1
// writes the pseudopotential psi = 1 - exp(-rho) of every node from its pulled
// density.  Pass 2 pulls again, adds the interaction force
// F = -G psi(x) sum_i w_i c_i psi(x + c_i) to the body force rho g (a
// neighbour behind a wall contributes the node's own psi), takes
// u = (sum f c + F/2)/rho and applies the forced central-moment collision of
// the single-phase step (Sec. II.B, Eq. eq:posColl0).
//
// The force needs psi at all 18 neighbours, and psi needs the neighbours'
// post-collision populations, so the step cannot be one pass without a halo
// exchange between thread blocks; psi costs 4 (8) bytes written and read per
// node.  Storage and initialisation are those of the single-phase step
// (f - w, FP64 or FP32).  Both phases sit far from the reference density, so
// the post-collision rest population is set from the mass balance
// (conserve_mass): without it FP32 repeats the same rounding error at every
// node of a uniform phase and loses about 2e-8 of density per node and step.
#include "lbm_internal.h"
#include "lbm_reduce.cuh"
#include "lbm_sc.cuh"

namespace lbm {

template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(256) sc_psi_kernel(const S* __restrict__ src, C* __restrict__ psi, ScArgs p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const Box& b = p.box;
    if (x >= b.nx) return;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q];
    gather19<S, C, WALLS>(src, b, q, x, y, z, self, (C)p.lid[0], (C)p.lid[1], (C)p.lid[2], f);
    psi[self] = pseudopotential<C>((C)1 + moments19(f).drho);
}

template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(256) sc_collide_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                         const C* __restrict__ psi, ScArgs p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const Box& b = p.box;
    if (x >= b.nx) return;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q];
    gather19<S, C, WALLS>(src, b, q, x, y, z, self, (C)p.lid[0], (C)p.lid[1], (C)p.lid[2], f);
    const Moments<C> m = moments19(f);
    const Macro<C> a = sc_macro<C>(m, psi, b, q, x, y, z, self, p);
    collide_fluid<C>(f, m, a, (C)p.omega);
    conserve_mass<C>(f, m.drho);
    scatter19<S, C>(dst, b.n, self, f);
}

// Fused step (launch variant 3): one kernel, psi kept on chip.  A CTA of
// 32 x BY threads covers an x-y tile of 30 x (BY - 2) nodes plus a one-node
// halo ring and marches through a chunk of lz planes.  For each plane z it
// pulls plane z + 1 at every tile and halo node, writes that plane's psi into a
// three-plane ring in shared memory, synchronises, and collides plane z at the
// tile nodes with psi of all 18 neighbours read from the ring; the populations
// of plane z + 1 stay in registers for the next plane.  psi never reaches HBM,
// so a step reads and writes the populations once (160 B/LUP algorithmic at
// FP32 becomes the traffic); the halo pulls are L2 hits of the neighbouring
// tiles' rows, and each chunk pulls its two end planes once more.
template <typename S, typename C, bool WALLS, int BY>
__global__ void __launch_bounds__(32 * BY) sc_fused_kernel(const S* __restrict__ src, S* __restrict__ dst, ScArgs p,
                                                           int lz) {
    constexpr int BX = 32, TX = BX - 2, TY = BY - 2;
    __shared__ C ring[3][BY][BX];
    const Box& b = p.box;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gx = (int)blockIdx.x * TX + tx - 1, gy = (int)blockIdx.y * TY + ty - 1;
    const int z0 = (int)blockIdx.z * lz, z1 = min(z0 + lz, b.nz);
    const bool px = b.periodic & 1u, py = b.periodic & 2u, pz = b.periodic & 4u;
    // this thread's node (wrapped on periodic axes; absent beyond a wall)
    int wx = gx, wy = gy;
    bool inside = true;
    if (gx < 0 || gx >= b.nx) {
        if (px)
            wx = ((gx % b.nx) + b.nx) % b.nx;
        else
            inside = false;
    }
    if (gy < 0 || gy >= b.ny) {
        if (py)
            wy = ((gy % b.ny) + b.ny) % b.ny;
        else
            inside = false;
    }
    const bool interior = tx >= 1 && tx <= TX && ty >= 1 && ty <= TY && gx < b.nx && gy < b.ny;
    const C lx = (C)p.lid[0], ly = (C)p.lid[1], lzv = (C)p.lid[2];
    auto pull = [&](int zz, C (&f)[Q]) {
        const Nbr q = make_nbr(b, wx, wy, zz);
        const uint32_t self = ((uint32_t)zz * (uint32_t)b.ny + (uint32_t)wy) * (uint32_t)b.nx + (uint32_t)wx;
        gather19<S, C, WALLS>(src, b, q, wx, wy, zz, self, lx, ly, lzv, f);
    };
    auto slot = [&](int zz) { return (zz - z0 + 1) % 3; };

    C f[Q];
    {
        const int zm = z0 - 1;
        if (inside && (zm >= 0 || pz)) {
            C t[Q];
            pull(zm >= 0 ? zm : zm + b.nz, t);
            ring[slot(zm)][ty][tx] = pseudopotential<C>((C)1 + moments19(t).drho);
        }
        if (inside) {
            C t[Q];
            pull(z0, t);
            ring[slot(z0)][ty][tx] = pseudopotential<C>((C)1 + moments19(t).drho);
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = t[i];
        }
    }
    for (int z = z0; z < z1; ++z) {
        const int zn = z + 1;
        C fn[Q];
        const bool next = inside && (zn < b.nz || pz);
        if (next) {
            pull(zn < b.nz ? zn : zn - b.nz, fn);
            ring[slot(zn)][ty][tx] = pseudopotential<C>((C)1 + moments19(fn).drho);
        }
        __syncthreads();
        if (interior) {
            const Nbr q = make_nbr(b, gx, gy, z);
            const int sm = slot(z - 1), s0 = slot(z), sp = slot(zn);
            const C own = ring[s0][ty][tx];
            C sx = (C)0, sy = (C)0, sz = (C)0;
#define LBM_SCF(I)                                                                                          \
    {                                                                                                       \
        constexpr int ex = cx_of(I), ey = cy_of(I), ez = cz_of(I);                                          \
        const bool wall = WALLS && ((ex > 0 && q.wxp) || (ex < 0 && q.wxm) || (ey > 0 && q.wyp) ||          \
                                    (ey < 0 && q.wym) || (ez > 0 && q.wzp) || (ez < 0 && q.wzm));           \
        const C t = (wall ? own : ring[ez == 0 ? s0 : (ez > 0 ? sp : sm)][ty + ey][tx + ex]) * (C)w_of(I);  \
        if (ex) sx += (C)ex * t;                                                                            \
        if (ey) sy += (C)ey * t;                                                                            \
        if (ez) sz += (C)ez * t;                                                                            \
    }
            LBM_SCF(1) LBM_SCF(2) LBM_SCF(3) LBM_SCF(4) LBM_SCF(5) LBM_SCF(6) LBM_SCF(7) LBM_SCF(8) LBM_SCF(9)
            LBM_SCF(10) LBM_SCF(11) LBM_SCF(12) LBM_SCF(13) LBM_SCF(14) LBM_SCF(15) LBM_SCF(16) LBM_SCF(17)
            LBM_SCF(18)
#undef LBM_SCF
            const Moments<C> m = moments19(f);
            Macro<C> a;
            a.rho = (C)1 + m.drho;
            const C mg = -(C)p.G * own;
            a.Fx = (a.rho * (C)p.g[0] - (C)p.rg[0]) + mg * sx;
            a.Fy = (a.rho * (C)p.g[1] - (C)p.rg[1]) + mg * sy;
            a.Fz = (a.rho * (C)p.g[2] - (C)p.rg[2]) + mg * sz;
            const C inv = recip(a.rho);
            a.ux = (m.jx + (C)0.5 * a.Fx) * inv;
            a.uy = (m.jy + (C)0.5 * a.Fy) * inv;
            a.uz = (m.jz + (C)0.5 * a.Fz) * inv;
            collide_fluid<C>(f, m, a, (C)p.omega);
            conserve_mass<C>(f, m.drho);
            const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)gy) * (uint32_t)b.nx + (uint32_t)gx;
            scatter19<S, C>(dst, b.n, self, f);
        }
        __syncthreads();
        if (next) {
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = fn[i];
        }
    }
}

// rho, u (with +F/2) and psi of a z-slab; psi of the whole box is current.
template <typename S, typename C, bool WALLS>
__global__ void sc_fields_kernel(const S* __restrict__ src, const C* __restrict__ psi, double* __restrict__ slab,
                                 ScArgs p, int z0, int nzs) {
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
    const Macro<C> a = sc_macro<C>(mo, psi, b, q, x, y, z, self, p);
    slab[k] = (double)a.rho;
    slab[m + k] = (double)a.ux;
    slab[2 * m + k] = (double)a.uy;
    slab[3 * m + k] = (double)a.uz;
    slab[4 * m + k] = (double)psi[self];
}

template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(RED_THREADS) sc_reduce_kernel(const S* __restrict__ src, const C* __restrict__ psi,
                                                                ScArgs p, C* __restrict__ uprev, bool have_prev,
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
            const Macro<C> a = sc_macro<C>(mo, psi, b, q, x, y, z, self, p);
            reduce_node<C>(acc, a.rho, a.ux, a.uy, a.uz, uprev, b.n, self, have_prev, record);
        }
    }
    block_reduce_store(acc, partials);
}

// ---------------------------------------------------------------------------
static ScArgs sc_args(const lbm_ctx* c) {
    ScArgs p;
    p.box = c->box;
    p.omega = c->relax.omega;
    p.G = c->phys.G;
    for (int a = 0; a < 3; ++a) {
        p.g[a] = c->forcing.g[a];
        p.rg[a] = c->forcing.rho_ref * c->forcing.g[a];
        p.lid[a] = (c->box.periodic & 2u) ? 0.0 : c->grid.lid_u[a];
    }
    return p;
}

template <typename S, typename C>
static void launch_psi(lbm_ctx* c, const S* src, const ScArgs& p) {
    const dim3 grid = step_grid(c->box, c->block_x);
    if ((c->box.periodic & 7u) != 7u)
        sc_psi_kernel<S, C, true><<<grid, c->block_x, 0, c->stream>>>(src, (C*)c->phi, p);
    else
        sc_psi_kernel<S, C, false><<<grid, c->block_x, 0, c->stream>>>(src, (C*)c->phi, p);
}

template <typename S, typename C, bool WALLS, int BY>
static void launch_fused(lbm_ctx* c, const S* src, S* dst, const ScArgs& p) {
    const int lz = c->zchunk > 0 ? c->zchunk : 32;
    const dim3 grid((unsigned)((c->box.nx + 29) / 30), (unsigned)((c->box.ny + BY - 3) / (BY - 2)),
                    (unsigned)((c->box.nz + lz - 1) / lz));
    sc_fused_kernel<S, C, WALLS, BY><<<grid, dim3(32, BY), 0, c->stream>>>(src, dst, p, lz);
}

template <typename S, typename C>
static cudaError_t step_t(lbm_ctx* c, long n, bool dry) {
    const ScArgs p = sc_args(c);
    const bool walls = (c->box.periodic & 7u) != 7u;
    const int bx = c->block_x;
    if (c->variant == 3) {
        const bool wide = c->fused_threads >= 512 && sizeof(C) == 4;
        for (long s = 0; s < n; ++s) {
            const S* src = (const S*)c->buf[c->cur];
            S* dst = (S*)c->buf[c->cur ^ 1];
            if (walls)
                wide ? launch_fused<S, C, true, 16>(c, src, dst, p) : launch_fused<S, C, true, 8>(c, src, dst, p);
            else
                wide ? launch_fused<S, C, false, 16>(c, src, dst, p) : launch_fused<S, C, false, 8>(c, src, dst, p);
            if (!dry) c->cur ^= 1;
        }
        return cudaGetLastError();
    }
    const dim3 grid = step_grid(c->box, bx);
    const C* psi = (const C*)c->phi;
    for (long s = 0; s < n; ++s) {
        const S* src = (const S*)c->buf[c->cur];
        S* dst = (S*)c->buf[c->cur ^ 1];
        launch_psi<S, C>(c, src, p);
        if (walls)
            sc_collide_kernel<S, C, true><<<grid, bx, 0, c->stream>>>(src, dst, psi, p);
        else
            sc_collide_kernel<S, C, false><<<grid, bx, 0, c->stream>>>(src, dst, psi, p);
        if (!dry) c->cur ^= 1;
    }
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t fields_t(lbm_ctx* c, double* slab, int z0, int nzs) {
    const ScArgs p = sc_args(c);
    const S* src = (const S*)c->buf[c->cur];
    if (z0 == 0) launch_psi<S, C>(c, src, p);  // slabs are read in order from z0 = 0
    const int bx = c->block_x;
    dim3 grid((unsigned)((c->box.nx + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)nzs);
    if ((c->box.periodic & 7u) != 7u)
        sc_fields_kernel<S, C, true><<<grid, bx, 0, c->stream>>>(src, (const C*)c->phi, slab, p, z0, nzs);
    else
        sc_fields_kernel<S, C, false><<<grid, bx, 0, c->stream>>>(src, (const C*)c->phi, slab, p, z0, nzs);
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t reduce_t(lbm_ctx* c, bool record) {
    const ScArgs p = sc_args(c);
    const S* src = (const S*)c->buf[c->cur];
    launch_psi<S, C>(c, src, p);
    if ((c->box.periodic & 7u) != 7u)
        sc_reduce_kernel<S, C, true><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            src, (const C*)c->phi, p, (C*)c->uprev, c->have_prev, record, c->partials);
    else
        sc_reduce_kernel<S, C, false><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            src, (const C*)c->phi, p, (C*)c->uprev, c->have_prev, record, c->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce_finalize(c);
}

cudaError_t sc_step(lbm_ctx* c, long n, bool dry) {
    return c->prec == LBM_FP64 ? step_t<double, double>(c, n, dry) : step_t<float, float>(c, n, dry);
}
cudaError_t sc_fields(lbm_ctx* c, double* slab, int z0, int nzs) {
    return c->prec == LBM_FP64 ? fields_t<double, double>(c, slab, z0, nzs) : fields_t<float, float>(c, slab, z0, nzs);
}
cudaError_t sc_reduce(lbm_ctx* c, bool record) {
    return c->prec == LBM_FP64 ? reduce_t<double, double>(c, record) : reduce_t<float, float>(c, record);
}

}  // namespace lbm
