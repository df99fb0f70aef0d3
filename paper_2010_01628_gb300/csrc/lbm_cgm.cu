// lbm_cgm.cu -- colour-gradient two-phase step (App. E of arXiv:2010.01628).
//
// Two passes per step.  Pass 1 pulls the populations of every node and writes
// the order parameter phi = (rho_r - rho_b)/(rho_r + rho_b) (Eq. eq:order) and
// the red density.  Pass 2 pulls again, collides the total populations in
// central-moment space toward h_eq (App. E post-collision list, with the 1/6 on
// k16..18 that makes it reduce to rho c_s^4 at alpha = 1/3), adds the
// surface-tension perturbation with the squared projection (c_i . grad phi)^2
// (the mass-conserving form of Eq. eq:perturb), and recolours (Eqs. eq:op3r,
// eq:op3b with g_eq(rho, 0) = rho phi_i(alpha)).  grad phi is the isotropic
// stencil (1/c_s^2) sum_i w_i c_i phi(x + c_i); a neighbour behind a wall
// contributes the node's own phi.
//
// Storage, 24 planes per copy, unshifted: 0..18 the total populations f_i;
// then, per node, the red fraction a = rho_r / rho and the recolouring vector
// V = beta (rho_r rho_b / rho) (1 - alpha) grad phi / |grad phi| of its last
// collision, and its red rest population.  The recolouring makes the red
// population of a moving direction a f_i + e_i with
// e_i = beta (rho_r rho_b / rho) cos(theta_i) phi_i(alpha) = kappa_i c_i . V
// (kappa = 1/12 on the axes, 1/(24 sqrt 2) on the diagonals), so it is rebuilt
// where it is pulled instead of stored, and blue is the total minus red: the
// state is 24 values per node instead of 38 (a step moves 284 B per node in
// FP32 instead of 464).
#include "lbm_internal.h"
#include "lbm_reduce.cuh"

namespace lbm {

struct CgmArgs {
    Box box;
    double omega, alpha_r, alpha_b, A, beta;
    double g[3];
    double rg[3];  // rho_ref g: F = rho g - rho_ref g
};

template <typename C>
struct CgmNode {
    C rho_r, rho_b, rho, ux, uy, uz, Fx, Fy, Fz, alpha;
};

constexpr int CGM_FRAC = Q, CGM_VX = Q + 1, CGM_VY = Q + 2, CGM_VZ = Q + 3, CGM_RED0 = Q + 4;

// Density of a population set: the 18 moving populations in direction order,
// then the rest population.  The stores below write the rest population as the
// density minus that same moving sum, so a uniform region sums back to its
// density (and its red density) exactly in FP32.
template <typename C>
__device__ __forceinline__ C colour_sum(const C (&f)[Q]) {
    C s = f[1];
#pragma unroll
    for (int i = 2; i < Q; ++i) s += f[i];
    return s + f[0];
}

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Red population of moving direction J at a node with red fraction a,
// recolouring vector V and total population f: a f + kappa_J c_J . V.  The
// collision that stores (f, a, V) and the pull that rebuilds it run this same
// sequence of roundings, so the red rest population stored for the mass
// balance matches the pulled red populations exactly.
template <typename C, int J>
__device__ __forceinline__ C red_pop(C a, C vx, C vy, C vz, C f) {
    constexpr int cx = cx_of(J), cy = cy_of(J), cz = cz_of(J);
    constexpr double kappa = cx * cx + cy * cy + cz * cz == 1 ? 1.0 / 12.0 : 0.70710678118654752440 / 24.0;
    C cv = (C)0;
    if (cx) cv = cx > 0 ? vx : -vx;
    if (cy) cv = cx ? (cy > 0 ? cv + vy : cv - vy) : (cy > 0 ? vy : -vy);
    if (cz) cv = (cx || cy) ? (cz > 0 ? cv + vz : cv - vz) : (cz > 0 ? vz : -vz);
    return fma_rn(a, f, (C)kappa * cv);
}

template <typename S, typename C>
__device__ __forceinline__ C cgm_ld(const S* __restrict__ src, size_t n, int plane, uint32_t cell) {
    return (C)Store<S>::load(src + (size_t)plane * n + cell);
}

// All 19 pulled populations of a node, f_I(x) = f*_I(x - c_I), and their red
// parts, rebuilt from the source node's red fraction and recolouring vector;
// from behind a wall, the node's own opposite direction (half-way bounce-back;
// the colour-gradient step has no moving lid).  Two phases: every load first
// (totals, and a and the needed components of V at the source nodes), then
// the red populations.
template <typename C>
struct RedSrc {
    C a, vx, vy, vz;
};
template <typename S, typename C, bool WALLS, int I>
__device__ __forceinline__ void cgm_load(const S* __restrict__ src, const Box& b, const Nbr& q, int x, int y, int z,
                                         uint32_t self, C& f, RedSrc<C>& g) {
    uint32_t cell;
    const bool wall = pull_source<I>(b, q, x, y, z, cell);
    constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
    const bool bb = WALLS && wall;
    const uint32_t at = bb ? self : cell;
    f = cgm_ld<S, C>(src, b.n, bb ? opp_of(I) : I, at);
    g.a = cgm_ld<S, C>(src, b.n, CGM_FRAC, at);
    g.vx = cx ? cgm_ld<S, C>(src, b.n, CGM_VX, at) : (C)0;
    g.vy = cy ? cgm_ld<S, C>(src, b.n, CGM_VY, at) : (C)0;
    g.vz = cz ? cgm_ld<S, C>(src, b.n, CGM_VZ, at) : (C)0;
}
template <typename S, typename C, bool WALLS>
__device__ __forceinline__ void cgm_pull_all(const S* __restrict__ src, const Box& b, const Nbr& q, int x, int y,
                                             int z, uint32_t self, C (&f)[Q], C (&r)[Q]) {
    RedSrc<C> g[Q];
    f[0] = cgm_ld<S, C>(src, b.n, 0, self);
    r[0] = cgm_ld<S, C>(src, b.n, CGM_RED0, self);
#define LBM_CL(I) cgm_load<S, C, WALLS, I>(src, b, q, x, y, z, self, f[I], g[I]);
    LBM_CL(1) LBM_CL(2) LBM_CL(3) LBM_CL(4) LBM_CL(5) LBM_CL(6) LBM_CL(7) LBM_CL(8) LBM_CL(9) LBM_CL(10)
    LBM_CL(11) LBM_CL(12) LBM_CL(13) LBM_CL(14) LBM_CL(15) LBM_CL(16) LBM_CL(17) LBM_CL(18)
#undef LBM_CL
    // a bounce-back pull takes the opposite direction's red part at the node
    // itself; c_opp = -c_I, so red_pop of I with -V equals red_pop of opp(I) with V
#define LBM_CR(I)                                                                                     \
    {                                                                                                 \
        uint32_t cell;                                                                                \
        const bool bb = WALLS && pull_source<I>(b, q, x, y, z, cell);                                 \
        r[I] = bb ? red_pop<C, opp_of(I)>(g[I].a, g[I].vx, g[I].vy, g[I].vz, f[I])                   \
                  : red_pop<C, I>(g[I].a, g[I].vx, g[I].vy, g[I].vz, f[I]);                           \
    }
    LBM_CR(1) LBM_CR(2) LBM_CR(3) LBM_CR(4) LBM_CR(5) LBM_CR(6) LBM_CR(7) LBM_CR(8) LBM_CR(9) LBM_CR(10)
    LBM_CR(11) LBM_CR(12) LBM_CR(13) LBM_CR(14) LBM_CR(15) LBM_CR(16) LBM_CR(17) LBM_CR(18)
#undef LBM_CR
}

// rho, F = rho g - rho_ref g and u = (sum f c + F/2)/rho of pulled totals
// (rho summed as colour_sum), with the colour densities rho_r and rho - rho_r.
template <typename C>
__device__ __forceinline__ CgmNode<C> cgm_macro(const C (&f)[Q], const Moments<C>& m, C rho_r, const CgmArgs& p) {
    CgmNode<C> s;
    s.rho = colour_sum(f);
    s.rho_r = rho_r;
    s.rho_b = s.rho - rho_r;
    s.Fx = s.rho * (C)p.g[0] - (C)p.rg[0];
    s.Fy = s.rho * (C)p.g[1] - (C)p.rg[1];
    s.Fz = s.rho * (C)p.g[2] - (C)p.rg[2];
    const C inv = recip(s.rho);
    s.ux = (m.jx + (C)0.5 * s.Fx) * inv;
    s.uy = (m.jy + (C)0.5 * s.Fy) * inv;
    s.uz = (m.jz + (C)0.5 * s.Fz) * inv;
    s.alpha = (s.rho_r * (C)p.alpha_r + s.rho_b * (C)p.alpha_b) * inv;
    return s;
}

// phi_i(alpha) of Eq. eq:varphi_ik.
template <typename C, int I>
__device__ __forceinline__ C cgm_phi_i(C alpha) {
    constexpr int n2 = cx_of(I) * cx_of(I) + cy_of(I) * cy_of(I) + cz_of(I) * cz_of(I);
    return n2 == 0 ? alpha : (n2 == 1 ? ((C)1 - alpha) * (C)(1.0 / 12.0) : ((C)1 - alpha) * (C)(1.0 / 24.0));
}

// Post-collision populations of the colour-gradient single-phase operator
// (kd = (1 - omega) k5..9 computed from raw moments as in the single-phase
// step; the equilibrated moments take App. E's values).
template <typename C>
__device__ __forceinline__ void cgm_collide(C (&f)[Q], const Moments<C>& m, const CgmNode<C>& s, C omega) {
    const C rho = s.rho, ux = s.ux, uy = s.uy, uz = s.uz, al = s.alpha;
    const C hx = (C)0.5 * s.Fx, hy = (C)0.5 * s.Fy, hz = (C)0.5 * s.Fz;
    const C om1 = (C)1 - omega;
    C kd[5];
    kd[0] = om1 * (m.pxx_m_pyy - rho * (ux * ux - uy * uy) + (C)2 * (ux * hx - uy * hy));
    kd[1] = om1 * (m.pyy_m_pzz - rho * (uy * uy - uz * uz) + (C)2 * (uy * hy - uz * hz));
    kd[2] = om1 * (m.pxy - rho * ux * uy + ux * hy + uy * hx);
    kd[3] = om1 * (m.pxz - rho * ux * uz + ux * hz + uz * hx);
    kd[4] = om1 * (m.pyz - rho * uy * uz + uy * hz + uz * hy);
    const C third = (C)(1.0 / 3.0);
    const C a3 = rho * ((C)3 * al - (C)1) * (C)(1.0 / 6.0);
    const C t[6] = {hy * third + a3 * uy, hx * third + a3 * ux, hz * third + a3 * uz,
                    hx * third + a3 * ux, hz * third + a3 * uz, hy * third + a3 * uy};
    const C k4 = (C)1.5 * rho * ((C)1 - al);
    const C x2 = ux * ux, y2 = uy * uy, z2 = uz * uz;
    const C sixth = (C)(1.0 / 6.0);
    const C k16 = rho * ((C)1 + x2 + y2 - al * ((C)1 + (C)3 * x2 + (C)3 * y2)) * sixth;
    const C k17 = rho * ((C)1 + x2 + z2 - al * ((C)1 + (C)3 * x2 + (C)3 * z2)) * sixth;
    const C k18 = rho * ((C)1 + y2 + z2 - al * ((C)1 + (C)3 * y2 + (C)3 * z2)) * sixth;
    back_transform<C>(rho, ux, uy, uz, hx, hy, hz, k4, rho, k4, kd, t, k16, k17, k18, f);
}

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

// grad phi = (1/c_s^2) sum_i w_i c_i phi(x + c_i): the axis and the diagonal
// neighbours are summed apart and scaled once (3/18 and 3/36).
template <typename C>
__device__ __forceinline__ void grad_phi(const C* __restrict__ phi, const Box& b, const Nbr& q, int x, int y, int z,
                                         uint32_t self, C (&gr)[3]) {
    const C own = phi[self];
    C ax = (C)0, ay = (C)0, az = (C)0, dx = (C)0, dy = (C)0, dz = (C)0;
#define LBM_GP(I)                                                                           \
    {                                                                                       \
        constexpr int ex = cx_of(I), ey = cy_of(I), ez = cz_of(I);                          \
        constexpr bool axis = ex * ex + ey * ey + ez * ez == 1;                             \
        const C t = field_nbr<C, I>(phi, b, q, x, y, z, own);                               \
        if (ex) { if (axis) ax += ex > 0 ? t : -t; else dx += ex > 0 ? t : -t; }            \
        if (ey) { if (axis) ay += ey > 0 ? t : -t; else dy += ey > 0 ? t : -t; }            \
        if (ez) { if (axis) az += ez > 0 ? t : -t; else dz += ez > 0 ? t : -t; }            \
    }
    LBM_GP(1) LBM_GP(2) LBM_GP(3) LBM_GP(4) LBM_GP(5) LBM_GP(6) LBM_GP(7) LBM_GP(8) LBM_GP(9) LBM_GP(10)
    LBM_GP(11) LBM_GP(12) LBM_GP(13) LBM_GP(14) LBM_GP(15) LBM_GP(16) LBM_GP(17) LBM_GP(18)
#undef LBM_GP
    const C wa = (C)(3.0 / 18.0), wd = (C)(3.0 / 36.0);
    gr[0] = wa * ax + wd * dx;
    gr[1] = wa * ay + wd * dy;
    gr[2] = wa * az + wd * dz;
}

// Direction I (1..18) after the collision: adds the perturbation, stores the
// total population and adds it and its red part to the running sums.
// pa = (A |grad phi| w_i / |grad phi|^2, A |grad phi| B_i) for the axis (index
// 0) and diagonal (index 1) weight classes; zero where |grad phi| vanishes.
template <typename S, typename C, int I>
__device__ __forceinline__ void perturb_store(S* __restrict__ dst, size_t n, uint32_t self, C fi, const C (&gr)[3],
                                              const C (&pa)[2][2], C a, const C (&v)[3], C& sum_f, C& sum_r) {
    constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
    constexpr int k = cx * cx + cy * cy + cz * cz == 1 ? 0 : 1;
    C cg = (C)0;
    if (cx) cg = cx > 0 ? gr[0] : -gr[0];
    if (cy) cg = cx ? (cy > 0 ? cg + gr[1] : cg - gr[1]) : (cy > 0 ? gr[1] : -gr[1]);
    if (cz) cg = (cx || cy) ? (cz > 0 ? cg + gr[2] : cg - gr[2]) : (cz > 0 ? gr[2] : -gr[2]);
    fi += pa[k][0] * (cg * cg) - pa[k][1];
    Store<S>::store(dst + (size_t)I * n + self, fi);
    const C ri = red_pop<C, I>(a, v[0], v[1], v[2], fi);
    if (I == 1) {
        sum_f = fi;
        sum_r = ri;
    } else {
        sum_f += fi;
        sum_r += ri;
    }
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
    mz.drho = mz.jx = mz.jy = mz.jz = (C)0;
    const C r = s.rho;
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
