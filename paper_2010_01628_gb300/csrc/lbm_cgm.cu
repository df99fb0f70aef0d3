// lbm_cgm.cu -- colour-gradient two-phase step (App. E of arXiv:2010.01628):
// the single-domain kernels (two passes per step), initialisation, fields and
// reductions.  The two passes take the same steps as cgm_phi_node and
// cgm_collide_node of lbm_cgm.cuh (which the batched persistent kernel uses),
// written out in the kernels: built on those node functions, the
// single-domain step compiled to code 8 % slower (16.9 against 18.5 GLUPS on
// the 256^3 droplets, GB300).
#include "lbm_cgm.cuh"
#include "lbm_internal.h"
#include "lbm_reduce.cuh"

namespace lbm {

// Pass 1: phi and rho_r of every node from its pulled populations.
template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(256) cgm_phi_kernel(const S* __restrict__ src, C* __restrict__ phi,
                                                      C* __restrict__ rho_red, CgmArgs p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const Box& b = p.box;
    if (x >= b.nx) return;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q], r[Q];
    cgm_pull_all<S, C, WALLS>(src, b, q, x, y, z, self, f, r);
    const C sr = colour_sum(r), st = colour_sum(f);
    phi[self] = (sr - (st - sr)) / st;
    rho_red[self] = sr;
}

// Pass 2: pull, collide the totals, perturb, recolour.
template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(256) cgm_collide_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                          const C* __restrict__ phi, const C* __restrict__ rho_red,
                                                          CgmArgs p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const Box& b = p.box;
    if (x >= b.nx) return;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q];
    gather19<S, C, WALLS>(src, b, q, x, y, z, self, (C)0, (C)0, (C)0, f);
    const Moments<C> m = moments19(f);
    const CgmNode<C> s = cgm_macro<C>(f, m, rho_red[self], p);
    cgm_collide<C>(f, m, s, (C)p.omega);
    C gr[3];
    grad_phi<C>(phi, b, q, x, y, z, self, gr);
    const C n2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
    const C nrm = sqrt(n2);
    // each colour's operator carries A_k/2 = A/2; together they perturb the total by
    // A |grad phi| (w_i (c_i . grad phi)^2 / |grad phi|^2 - B_i), B = 1/18, 1/36
    const C pert_amp = n2 > (C)1e-24 ? (C)p.A * nrm : (C)0;
    const C pq = pert_amp * (n2 > (C)1e-24 ? recip(n2) : (C)0);
    const C pa[2][2] = {{pq * (C)(1.0 / 18.0), pert_amp * (C)(1.0 / 18.0)},
                        {pq * (C)(1.0 / 36.0), pert_amp * (C)(1.0 / 36.0)}};
    const C inv_nrm = nrm > (C)1e-12 ? recip(nrm) : (C)0;
    const C inv_rho = recip(s.rho);
    // recolouring: red fraction rho_r / rho, and V = beta rho_r rho_b / rho (1 - alpha) grad phi / |grad phi|
    const C a = s.rho_r * inv_rho;
    const C w = (C)p.beta * s.rho_r * s.rho_b * inv_rho * ((C)1 - s.alpha) * inv_nrm;
    const C v[3] = {w * gr[0], w * gr[1], w * gr[2]};
    C sum_f, sum_r;
#define LBM_PS(I) perturb_store<S, C, I>(dst, b.n, self, f[I], gr, pa, a, v, sum_f, sum_r);
    LBM_PS(1) LBM_PS(2) LBM_PS(3) LBM_PS(4) LBM_PS(5) LBM_PS(6) LBM_PS(7) LBM_PS(8) LBM_PS(9)
    LBM_PS(10) LBM_PS(11) LBM_PS(12) LBM_PS(13) LBM_PS(14) LBM_PS(15) LBM_PS(16) LBM_PS(17) LBM_PS(18)
#undef LBM_PS
    // Rest direction from the mass balances (the perturbation and the
    // recolouring conserve each colour; cos(theta_0) = 0).
    Store<S>::store(dst + self, s.rho - sum_f);
    Store<S>::store(dst + (size_t)CGM_RED0 * b.n + self, s.rho_r - sum_r);
    Store<S>::store(dst + (size_t)CGM_FRAC * b.n + self, a);
    Store<S>::store(dst + (size_t)CGM_VX * b.n + self, v[0]);
    Store<S>::store(dst + (size_t)CGM_VY * b.n + self, v[1]);
    Store<S>::store(dst + (size_t)CGM_VZ * b.n + self, v[2]);
}

template <typename S, typename C>
__global__ void cgm_init_kernel(S* __restrict__ dst, const double* __restrict__ slab, CgmArgs p, int z0, int nzs,
                                bool uniform) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, zs = blockIdx.z;
    const Box& b = p.box;
    if (x >= b.nx || zs >= nzs) return;
    const size_t m = (size_t)b.nx * b.ny * nzs;
    const size_t k = ((size_t)zs * b.ny + y) * b.nx + x;
    const uint32_t self = ((uint32_t)(z0 + zs) * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    double rho = 1.0, ph = -1.0;
    CgmNode<C> s;
    s.ux = s.uy = s.uz = (C)0;
    if (!uniform) {
        rho = slab[k];
        ph = slab[4 * m + k];
        s.ux = (C)slab[m + k];
        s.uy = (C)slab[2 * m + k];
        s.uz = (C)slab[3 * m + k];
    }
    const double rr = rho * (1.0 + ph) * 0.5, rb = rho * (1.0 - ph) * 0.5;
    s.rho_r = (C)rr;
    s.rho_b = (C)rb;
    s.rho = (C)rho;
    s.Fx = s.Fy = s.Fz = (C)0;
    s.alpha = (C)((rr * p.alpha_r + rb * p.alpha_b) / rho);
    // h_eq = T^-1 k_eq: the CGM collision of a state with zero deviatoric CMs
    Moments<C> mz;
    const C r = s.rho;
    // unforced: the momentum sum f c = rho u is the collision's r1..3*
    mz.drho = (C)0;
    mz.jx = r * s.ux;
    mz.jy = r * s.uy;
    mz.jz = r * s.uz;
    mz.pxx_m_pyy = r * (s.ux * s.ux - s.uy * s.uy);
    mz.pyy_m_pzz = r * (s.uy * s.uy - s.uz * s.uz);
    mz.pxy = r * s.ux * s.uy;
    mz.pxz = r * s.ux * s.uz;
    mz.pyz = r * s.uy * s.uz;
    C h[Q];
    cgm_collide<C>(h, mz, s, (C)0);  // omega = 0 keeps kd = k5..9 = 0 exactly
    // each colour takes its density fraction of h_eq: red fraction rr / rho, V = 0
    const C a = (C)(rr / rho), zero = (C)0;
    const C v[3] = {zero, zero, zero};
    const C pa[2][2] = {{zero, zero}, {zero, zero}};
    C sum_f, sum_r;
#define LBM_IS(I) perturb_store<S, C, I>(dst, b.n, self, h[I], v, pa, a, v, sum_f, sum_r);
    LBM_IS(1) LBM_IS(2) LBM_IS(3) LBM_IS(4) LBM_IS(5) LBM_IS(6) LBM_IS(7) LBM_IS(8) LBM_IS(9)
    LBM_IS(10) LBM_IS(11) LBM_IS(12) LBM_IS(13) LBM_IS(14) LBM_IS(15) LBM_IS(16) LBM_IS(17) LBM_IS(18)
#undef LBM_IS
    Store<S>::store(dst + self, s.rho - sum_f);
    Store<S>::store(dst + (size_t)CGM_RED0 * b.n + self, s.rho_r - sum_r);
    Store<S>::store(dst + (size_t)CGM_FRAC * b.n + self, a);
    Store<S>::store(dst + (size_t)CGM_VX * b.n + self, zero);
    Store<S>::store(dst + (size_t)CGM_VY * b.n + self, zero);
    Store<S>::store(dst + (size_t)CGM_VZ * b.n + self, zero);
}

template <typename S, typename C, bool WALLS>
__global__ void cgm_fields_kernel(const S* __restrict__ src, double* __restrict__ slab, CgmArgs p, int z0, int nzs) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, zs = blockIdx.z;
    const Box& b = p.box;
    if (x >= b.nx || zs >= nzs) return;
    const int z = z0 + zs;
    const size_t m = (size_t)b.nx * b.ny * nzs;
    const size_t k = ((size_t)zs * b.ny + y) * b.nx + x;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q], r[Q];
    cgm_pull_all<S, C, WALLS>(src, b, q, x, y, z, self, f, r);
    const Moments<C> mo = moments19(f);
    const CgmNode<C> s = cgm_macro<C>(f, mo, colour_sum(r), p);
    slab[k] = (double)s.rho;
    slab[m + k] = (double)s.ux;
    slab[2 * m + k] = (double)s.uy;
    slab[3 * m + k] = (double)s.uz;
    slab[4 * m + k] = (double)((s.rho_r - s.rho_b) / s.rho);
}

template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(RED_THREADS) cgm_reduce_kernel(const S* __restrict__ src, CgmArgs p,
                                                                 C* __restrict__ uprev, bool have_prev, bool record,
                                                                 double* __restrict__ partials) {
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
            gather19<S, C, WALLS>(src, b, q, x, y, z, self, (C)0, (C)0, (C)0, f);
            const Moments<C> mo = moments19(f);
            // rho and u need only the totals (the force is rho g - rho_ref g)
            const CgmNode<C> s = cgm_macro<C>(f, mo, (C)0, p);
            reduce_node<C>(acc, s.rho, s.ux, s.uy, s.uz, uprev, b.n, self, have_prev, record);
        }
    }
    block_reduce_store(acc, partials);
}

// ---------------------------------------------------------------------------
static CgmArgs cgm_args(const lbm_ctx* c) {
    CgmArgs p;
    p.box = c->box;
    p.omega = c->relax.omega;
    p.alpha_r = c->phys.alpha_r;
    p.alpha_b = c->phys.alpha_b;
    p.A = c->phys.A;
    p.beta = c->phys.beta;
    for (int a = 0; a < 3; ++a) {
        p.g[a] = c->forcing.g[a];
        p.rg[a] = c->forcing.rho_ref * c->forcing.g[a];
    }
    return p;
}

template <typename S, typename C>
static cudaError_t step_t(lbm_ctx* c, long n, bool dry) {
    const CgmArgs p = cgm_args(c);
    const bool walls = (c->box.periodic & 7u) != 7u;
    const int bx = c->block_x;
    const dim3 grid = step_grid(c->box, bx);
    C* phi = (C*)c->phi;
    C* rho_red = phi + c->box.n;  // the second scratch plane
    for (long s = 0; s < n; ++s) {
        const S* src = (const S*)c->buf[c->cur];
        S* dst = (S*)c->buf[c->cur ^ 1];
        if (walls) {
            cgm_phi_kernel<S, C, true><<<grid, bx, 0, c->stream>>>(src, phi, rho_red, p);
            cgm_collide_kernel<S, C, true><<<grid, bx, 0, c->stream>>>(src, dst, phi, rho_red, p);
        } else {
            cgm_phi_kernel<S, C, false><<<grid, bx, 0, c->stream>>>(src, phi, rho_red, p);
            cgm_collide_kernel<S, C, false><<<grid, bx, 0, c->stream>>>(src, dst, phi, rho_red, p);
        }
        if (!dry) c->cur ^= 1;
    }
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t init_t(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform) {
    const int bx = c->block_x;
    dim3 grid((unsigned)((c->box.nx + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)nzs);
    cgm_init_kernel<S, C><<<grid, bx, 0, c->stream>>>((S*)c->buf[c->cur], slab, cgm_args(c), z0, nzs, uniform);
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t fields_t(lbm_ctx* c, double* slab, int z0, int nzs) {
    const CgmArgs p = cgm_args(c);
    const int bx = c->block_x;
    dim3 grid((unsigned)((c->box.nx + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)nzs);
    if ((c->box.periodic & 7u) != 7u)
        cgm_fields_kernel<S, C, true><<<grid, bx, 0, c->stream>>>((const S*)c->buf[c->cur], slab, p, z0, nzs);
    else
        cgm_fields_kernel<S, C, false><<<grid, bx, 0, c->stream>>>((const S*)c->buf[c->cur], slab, p, z0, nzs);
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t reduce_t(lbm_ctx* c, bool record) {
    const CgmArgs p = cgm_args(c);
    if ((c->box.periodic & 7u) != 7u)
        cgm_reduce_kernel<S, C, true><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            (const S*)c->buf[c->cur], p, (C*)c->uprev, c->have_prev, record, c->partials);
    else
        cgm_reduce_kernel<S, C, false><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            (const S*)c->buf[c->cur], p, (C*)c->uprev, c->have_prev, record, c->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce_finalize(c);
}

cudaError_t cgm_step(lbm_ctx* c, long n, bool dry) {
    return c->prec == LBM_FP64 ? step_t<double, double>(c, n, dry) : step_t<float, float>(c, n, dry);
}
cudaError_t cgm_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform) {
    return c->prec == LBM_FP64 ? init_t<double, double>(c, slab, z0, nzs, uniform)
                               : init_t<float, float>(c, slab, z0, nzs, uniform);
}
cudaError_t cgm_fields(lbm_ctx* c, double* slab, int z0, int nzs) {
    return c->prec == LBM_FP64 ? fields_t<double, double>(c, slab, z0, nzs) : fields_t<float, float>(c, slab, z0, nzs);
}
cudaError_t cgm_reduce(lbm_ctx* c, bool record) {
    return c->prec == LBM_FP64 ? reduce_t<double, double>(c, record) : reduce_t<float, float>(c, record);
}

}  // namespace lbm
