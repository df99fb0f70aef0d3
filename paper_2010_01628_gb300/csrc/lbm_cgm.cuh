// lbm_cgm.cuh -- device side of the colour-gradient two-phase step (App. E of
// arXiv:2010.01628): the pull, moments, collision, gradient, perturbation and
// recolouring shared by the single-domain kernels (lbm_cgm.cu) and the
// batched persistent kernel (lbm_batch.cu), and the node functions of the two
// passes that the batch runs.
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
#pragma once

#include "lbm_device.cuh"

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

// NC: read-only path; else a plain cached load (persistent kernels whose
// sources are rewritten between grid-wide barriers).
template <typename S, typename C, bool NC = true>
__device__ __forceinline__ C cgm_ld(const S* __restrict__ src, size_t n, int plane, uint32_t cell) {
    if (NC) return (C)Store<S>::load(src + (size_t)plane * n + cell);
    return (C)Store<S>::load_coherent(src + (size_t)plane * n + cell);
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
template <typename S, typename C, bool WALLS, int I, bool NC = true>
__device__ __forceinline__ void cgm_load(const S* __restrict__ src, const Box& b, const Nbr& q, int x, int y, int z,
                                         uint32_t self, C& f, RedSrc<C>& g) {
    uint32_t cell;
    const bool wall = pull_source<I>(b, q, x, y, z, cell);
    constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
    const bool bb = WALLS && wall;
    const uint32_t at = bb ? self : cell;
    f = cgm_ld<S, C, NC>(src, b.n, bb ? opp_of(I) : I, at);
    g.a = cgm_ld<S, C, NC>(src, b.n, CGM_FRAC, at);
    g.vx = cx ? cgm_ld<S, C, NC>(src, b.n, CGM_VX, at) : (C)0;
    g.vy = cy ? cgm_ld<S, C, NC>(src, b.n, CGM_VY, at) : (C)0;
    g.vz = cz ? cgm_ld<S, C, NC>(src, b.n, CGM_VZ, at) : (C)0;
}
template <typename S, typename C, bool WALLS, bool NC = true>
__device__ __forceinline__ void cgm_pull_all(const S* __restrict__ src, const Box& b, const Nbr& q, int x, int y,
                                             int z, uint32_t self, C (&f)[Q], C (&r)[Q]) {
    RedSrc<C> g[Q];
    f[0] = cgm_ld<S, C, NC>(src, b.n, 0, self);
    r[0] = cgm_ld<S, C, NC>(src, b.n, CGM_RED0, self);
#define LBM_CL(I) cgm_load<S, C, WALLS, I, NC>(src, b, q, x, y, z, self, f[I], g[I]);
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
    back_transform<C>(rho, ux, uy, uz, hx, hy, hz, m.jx + s.Fx, m.jy + s.Fy, m.jz + s.Fz, k4, rho, k4, kd, t, k16,
                      k17, k18, f);
}

// Pass 1 at one node: phi and rho_r from its pulled populations.
template <typename S, typename C, bool WALLS, bool NC>
__device__ __forceinline__ void cgm_phi_node(const S* __restrict__ src, C* __restrict__ phi, C* __restrict__ rho_red,
                                             const CgmArgs& p, int x, int y, int z) {
    const Box& b = p.box;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q], r[Q];
    cgm_pull_all<S, C, WALLS, NC>(src, b, q, x, y, z, self, f, r);
    const C sr = colour_sum(r), st = colour_sum(f);
    phi[self] = (sr - (st - sr)) / st;
    rho_red[self] = sr;
}

// grad phi = (1/c_s^2) sum_i w_i c_i phi(x + c_i): the axis and the diagonal
// neighbours are summed apart and scaled once (3/18 and 3/36).
template <typename C, bool NC = true>
__device__ __forceinline__ void grad_phi(const C* __restrict__ phi, const Box& b, const Nbr& q, int x, int y, int z,
                                         uint32_t self, C (&gr)[3]) {
    const C own = NC ? phi[self] : ld_coherent(phi + self);
    C ax = (C)0, ay = (C)0, az = (C)0, dx = (C)0, dy = (C)0, dz = (C)0;
#define LBM_GP(I)                                                                           \
    {                                                                                       \
        constexpr int ex = cx_of(I), ey = cy_of(I), ez = cz_of(I);                          \
        constexpr bool axis = ex * ex + ey * ey + ez * ez == 1;                             \
        const C t = field_nbr<C, I, NC>(phi, b, q, x, y, z, own);                           \
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

// Pass 2 at one node: pull, collide the totals, perturb, recolour.
template <typename S, typename C, bool WALLS, bool NC>
__device__ __forceinline__ void cgm_collide_node(const S* __restrict__ src, S* __restrict__ dst,
                                                 const C* __restrict__ phi, const C* __restrict__ rho_red,
                                                 const CgmArgs& p, int x, int y, int z) {
    const Box& b = p.box;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q];
    gather19<S, C, WALLS, NC>(src, b, q, x, y, z, self, (C)0, (C)0, (C)0, f);
    const Moments<C> m = moments19(f);
    const CgmNode<C> s = cgm_macro<C>(f, m, NC ? rho_red[self] : ld_coherent(rho_red + self), p);
    cgm_collide<C>(f, m, s, (C)p.omega);
    C gr[3];
    grad_phi<C, NC>(phi, b, q, x, y, z, self, gr);
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

}  // namespace lbm
