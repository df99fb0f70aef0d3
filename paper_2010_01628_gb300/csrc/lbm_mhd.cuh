// lbm_mhd.cuh -- per-node magnetohydrodynamic update (Sec. III.F of
// arXiv:2010.01628), shared by the single-domain and batched kernels.
//
// The paper defers the magnetic solver to Dellar (2002).  Reading used here:
// BGK populations g_{m,a} on D3Q7 (rest + 6 axis directions), b = sum_m g_m,
// equilibrium w_m [b_a + c_{m,b} (u_b b_a - b_b u_a) / cs_m^2] with w = 1/4,
// 1/8 and cs_m^2 = 1/4, so eta = (tau_m - 1/2)/4.  The current density comes
// from the antisymmetric part of the non-equilibrium flux,
// j_c = -eps_{cba} (Lambda - Lambda_eq)_{ba} / (tau_m cs_m^2), with Lambda_eq
// evaluated at the unforced velocity sum f c / rho.  Walls impose b = b_wall
// by anti-bounce-back.
//
// State layout: planes 0..18 hold the shifted fluid populations, planes
// 19 + 3m + a the magnetic population of direction m, component a.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

struct MhdArgs {
    Box box;
    double omega, inv_tau_m, tau_m;
    double jfac;  // 1 / (tau_m c_s,m^2), the factor of the current density
    double g[3];
    double bw[3];
};

__host__ __device__ constexpr int mcx(int m) { return m == 1 ? 1 : (m == 2 ? -1 : 0); }
__host__ __device__ constexpr int mcy(int m) { return m == 3 ? 1 : (m == 4 ? -1 : 0); }
__host__ __device__ constexpr int mcz(int m) { return m == 5 ? 1 : (m == 6 ? -1 : 0); }
__host__ __device__ constexpr int mopp(int m) { return m == 0 ? 0 : ((m & 1) ? m + 1 : m - 1); }
__host__ __device__ constexpr double mw(int m) { return m == 0 ? 0.25 : 0.125; }
constexpr double CSM2 = 0.25;

template <typename S, typename C, bool WALLS, int M, bool NC>
__device__ __forceinline__ void gather_mag_dir(const S* __restrict__ gsrc, const Box& b, const Nbr& q, int x, int y,
                                               int z, uint32_t self, const C (&bw)[3], C (&g)[7][3]) {
    constexpr int cx = mcx(M), cy = mcy(M), cz = mcz(M);
    const int sx = cx == 0 ? x : (cx > 0 ? q.xm : q.xp);
    const int sy = cy == 0 ? y : (cy > 0 ? q.ym : q.yp);
    const int sz = cz == 0 ? z : (cz > 0 ? q.zm : q.zp);
    const bool wall = (cx > 0 && q.wxm) || (cx < 0 && q.wxp) || (cy > 0 && q.wym) || (cy < 0 && q.wyp) ||
                      (cz > 0 && q.wzm) || (cz < 0 && q.wzp);
    const uint32_t cell = ((uint32_t)sz * (uint32_t)b.ny + (uint32_t)sy) * (uint32_t)b.nx + (uint32_t)sx;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const S* p = (!WALLS || !wall) ? gsrc + (size_t)(3 * M + a) * b.n + cell
                                       : gsrc + (size_t)(3 * mopp(M) + a) * b.n + self;
        const C v = NC ? (C)Store<S>::load(p) : (C)Store<S>::load_coherent(p);
        g[M][a] = (!WALLS || !wall) ? v : -v + (C)(2.0 * mw(M)) * bw[a];
    }
}

template <typename S, typename C, bool WALLS, bool NC = true>
__device__ __forceinline__ void gather_mag(const S* __restrict__ gsrc, const Box& b, const Nbr& q, int x, int y,
                                           int z, uint32_t self, const C (&bw)[3], C (&g)[7][3]) {
    gather_mag_dir<S, C, WALLS, 0, NC>(gsrc, b, q, x, y, z, self, bw, g);
    gather_mag_dir<S, C, WALLS, 1, NC>(gsrc, b, q, x, y, z, self, bw, g);
    gather_mag_dir<S, C, WALLS, 2, NC>(gsrc, b, q, x, y, z, self, bw, g);
    gather_mag_dir<S, C, WALLS, 3, NC>(gsrc, b, q, x, y, z, self, bw, g);
    gather_mag_dir<S, C, WALLS, 4, NC>(gsrc, b, q, x, y, z, self, bw, g);
    gather_mag_dir<S, C, WALLS, 5, NC>(gsrc, b, q, x, y, z, self, bw, g);
    gather_mag_dir<S, C, WALLS, 6, NC>(gsrc, b, q, x, y, z, self, bw, g);
}

// b, the Lorentz force and the corrected velocity of one node.
template <typename C>
__device__ __forceinline__ Macro<C> mhd_macro(const Moments<C>& m, const C (&g)[7][3], const MhdArgs& p, C (&bb)[3]) {
    Macro<C> a;
    a.rho = (C)1 + m.drho;
    const C inv = recip(a.rho);
    const C us[3] = {m.jx * inv, m.jy * inv, m.jz * inv};
#pragma unroll
    for (int k = 0; k < 3; ++k) bb[k] = g[0][k] + g[1][k] + g[2][k] + g[3][k] + g[4][k] + g[5][k] + g[6][k];
    // non-equilibrium flux N_{ba} = sum_m c_{m,b} g_{m,a} - (u_b b_a - b_b u_a)
    C N[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        N[0][k] = (g[1][k] - g[2][k]) - (us[0] * bb[k] - bb[0] * us[k]);
        N[1][k] = (g[3][k] - g[4][k]) - (us[1] * bb[k] - bb[1] * us[k]);
        N[2][k] = (g[5][k] - g[6][k]) - (us[2] * bb[k] - bb[2] * us[k]);
    }
    const C s = -(C)p.jfac;
    const C jx = s * (N[1][2] - N[2][1]);
    const C jy = s * (N[2][0] - N[0][2]);
    const C jz = s * (N[0][1] - N[1][0]);
    a.Fx = a.rho * (C)p.g[0] + (jy * bb[2] - jz * bb[1]);
    a.Fy = a.rho * (C)p.g[1] + (jz * bb[0] - jx * bb[2]);
    a.Fz = a.rho * (C)p.g[2] + (jx * bb[1] - jy * bb[0]);
    a.ux = (m.jx + (C)0.5 * a.Fx) * inv;
    a.uy = (m.jy + (C)0.5 * a.Fy) * inv;
    a.uz = (m.jz + (C)0.5 * a.Fz) * inv;
    return a;
}

template <typename C, int M>
__device__ __forceinline__ C geq(int k, C ux, C uy, C uz, const C (&bb)[3]) {
    const C u[3] = {ux, uy, uz};
    C v = bb[k];
    if (mcx(M)) v += (C)(mcx(M) / CSM2) * (u[0] * bb[k] - bb[0] * u[k]);
    if (mcy(M)) v += (C)(mcy(M) / CSM2) * (u[1] * bb[k] - bb[1] * u[k]);
    if (mcz(M)) v += (C)(mcz(M) / CSM2) * (u[2] * bb[k] - bb[2] * u[k]);
    return (C)mw(M) * v;
}

template <typename S, typename C, int M>
__device__ __forceinline__ void relax_store_mag(S* __restrict__ gdst, size_t n, uint32_t self, const C (&g)[7][3],
                                                const Macro<C>& a, const C (&bb)[3], C inv_tau) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const C e = geq<C, M>(k, a.ux, a.uy, a.uz, bb);
        Store<S>::store(gdst + (size_t)(3 * M + k) * n + self, g[M][k] - (g[M][k] - e) * inv_tau);
    }
}

template <typename S, typename C, int M>
__device__ __forceinline__ void store_geq(S* __restrict__ gdst, size_t n, uint32_t self, C ux, C uy, C uz,
                                          const C (&bb)[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) Store<S>::store(gdst + (size_t)(3 * M + k) * n + self, geq<C, M>(k, ux, uy, uz, bb));
}

// One node: fluid and magnetic pulls, Lorentz force, CM collision, magnetic
// BGK, stores.
template <typename S, typename C, bool WALLS, bool NC>
__device__ __forceinline__ void mhd_node(const S* __restrict__ src, S* __restrict__ dst, const MhdArgs& p, int x,
                                         int y, int z) {
    const Box& b = p.box;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q];
    gather19<S, C, WALLS, NC>(src, b, q, x, y, z, self, (C)0, (C)0, (C)0, f);
    const C bw[3] = {(C)p.bw[0], (C)p.bw[1], (C)p.bw[2]};
    C g[7][3];
    gather_mag<S, C, WALLS, NC>(src + (size_t)Q * b.n, b, q, x, y, z, self, bw, g);
    const Moments<C> m = moments19(f);
    C bb[3];
    const Macro<C> a = mhd_macro<C>(m, g, p, bb);
    collide_fluid<C>(f, m, a, (C)p.omega);
    scatter19<S, C>(dst, b.n, self, f);
    S* gdst = dst + (size_t)Q * b.n;
    const C it = (C)p.inv_tau_m;
    relax_store_mag<S, C, 0>(gdst, b.n, self, g, a, bb, it);
    relax_store_mag<S, C, 1>(gdst, b.n, self, g, a, bb, it);
    relax_store_mag<S, C, 2>(gdst, b.n, self, g, a, bb, it);
    relax_store_mag<S, C, 3>(gdst, b.n, self, g, a, bb, it);
    relax_store_mag<S, C, 4>(gdst, b.n, self, g, a, bb, it);
    relax_store_mag<S, C, 5>(gdst, b.n, self, g, a, bb, it);
    relax_store_mag<S, C, 6>(gdst, b.n, self, g, a, bb, it);
}

}  // namespace lbm
