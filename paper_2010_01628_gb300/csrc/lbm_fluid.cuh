// lbm_fluid.cuh -- per-node single-phase update (Sec. II of arXiv:2010.01628),
// shared by the single-domain kernels and the batched persistent kernel.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

struct FluidArgs {
    Box box;
    double omega;
    double g[3];
    double lid[3];
};

template <typename C>
__device__ __forceinline__ Macro<C> fluid_macro(const Moments<C>& m, C gx, C gy, C gz) {
    Macro<C> a;
    a.rho = (C)1 + m.drho;
    a.Fx = a.rho * gx;  // F = rho g
    a.Fy = a.rho * gy;
    a.Fz = a.rho * gz;
    const C inv = recip(a.rho);
    a.ux = (m.jx + (C)0.5 * a.Fx) * inv;
    a.uy = (m.jy + (C)0.5 * a.Fy) * inv;
    a.uz = (m.jz + (C)0.5 * a.Fz) * inv;
    return a;
}

// Regularized on-node wall (Latt, Chopard, Malaspinas, Deville and Michler,
// Phys. Rev. E 77, 056703 (2008), the walls the paper imposes) on a y boundary
// node; SGN = +1 at y = 0, -1 at y = ny - 1 (the inward normal's y component).
// f holds the pulled shifted populations f - w; the five with c_y = SGN came
// from beyond the wall and are rebuilt:
//   rho (1 - u_n + g_n/2) = rho_0 + 2 rho_out from the known ones (the bare
//   normal momentum is rho u_n - F_n/2 with F = rho g); u_eq = u_w - g/2 so the
//   corrected velocity is u_w; unknowns by bounce-back of f - f_eq; then every
//   population becomes f_eq + w_i/(2 c_s^4) Q_i : Pi_neq.
template <typename C, int SGN>
__device__ __forceinline__ void regularize_wall(C (&f)[Q], C uwx, C uwy, C uwz, C gx, C gy, C gz) {
    C s0 = (C)0, sout = (C)0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (cy_of(i) == 0) s0 += f[i];
        if (cy_of(i) == -SGN) sout += f[i];
    }
    const C un = (C)SGN * uwy, gn = (C)SGN * gy;
    const C den = (C)1 - un + (C)0.5 * gn;
    // shifted: the weights of c_y = 0 plus twice those of c_y = -SGN sum to 1
    const C drho = (s0 + (C)2 * sout + un - (C)0.5 * gn) / den;
    const C rho = (C)1 + drho;
    C feq[Q];
    equilibrium_shifted<C>(rho, drho, uwx - (C)0.5 * gx, uwy - (C)0.5 * gy, uwz - (C)0.5 * gz, feq);
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (cy_of(i) == SGN) f[i] = feq[i] + (f[opp_of(i)] - feq[opp_of(i)]);
    C pxx = (C)0, pyy = (C)0, pzz = (C)0, pxy = (C)0, pxz = (C)0, pyz = (C)0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const C d = f[i] - feq[i];
        if (cx_of(i)) pxx += d;
        if (cy_of(i)) pyy += d;
        if (cz_of(i)) pzz += d;
        if (cx_of(i) * cy_of(i)) pxy += (C)(cx_of(i) * cy_of(i)) * d;
        if (cx_of(i) * cz_of(i)) pxz += (C)(cx_of(i) * cz_of(i)) * d;
        if (cy_of(i) * cz_of(i)) pyz += (C)(cy_of(i) * cz_of(i)) * d;
    }
    const C tr3 = (pxx + pyy + pzz) * (C)(1.0 / 3.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        C qp = -tr3;
        if (cx_of(i)) qp += pxx;
        if (cy_of(i)) qp += pyy;
        if (cz_of(i)) qp += pzz;
        if (cx_of(i) * cy_of(i)) qp += (C)(2 * cx_of(i) * cy_of(i)) * pxy;
        if (cx_of(i) * cz_of(i)) qp += (C)(2 * cx_of(i) * cz_of(i)) * pxz;
        if (cy_of(i) * cz_of(i)) qp += (C)(2 * cy_of(i) * cz_of(i)) * pyz;
        f[i] = feq[i] + (C)(4.5 * w_of(i)) * qp;
    }
}

// Pull of one node with regularized walls on y (x and z periodic): the wall
// rows rebuild the populations that came through the wall.
template <typename S, typename C>
__device__ __forceinline__ void gather_regularized(const S* __restrict__ src, const FluidArgs& p, const Nbr& q, int x,
                                                   int y, int z, uint32_t self, C (&f)[Q]) {
    const Box& b = p.box;
    gather19<S, C, true>(src, b, q, x, y, z, self, (C)0, (C)0, (C)0, f);
    if (y == 0)
        regularize_wall<C, 1>(f, (C)0, (C)0, (C)0, (C)p.g[0], (C)p.g[1], (C)p.g[2]);
    else if (y == b.ny - 1)
        regularize_wall<C, -1>(f, (C)p.lid[0], (C)p.lid[1], (C)p.lid[2], (C)p.g[0], (C)p.g[1], (C)p.g[2]);
}

// One node: pull (stream + boundaries), moments, forced CM collision, store.
// NC selects the read-only load path (sources not written during the kernel);
// RM the raw-moment variant of App. C.
template <typename S, typename C, bool WALLS, bool NC, bool RM = false>
__device__ __forceinline__ void fluid_node(const S* __restrict__ src, S* __restrict__ dst, const FluidArgs& p, int x,
                                           int y, int z) {
    const Box& b = p.box;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q];
    gather19<S, C, WALLS, NC>(src, b, q, x, y, z, self, (C)p.lid[0], (C)p.lid[1], (C)p.lid[2], f);
    const Moments<C> m = moments19(f);
    const Macro<C> a = fluid_macro(m, (C)p.g[0], (C)p.g[1], (C)p.g[2]);
    if (RM)
        collide_fluid_rm<C>(f, m, a, (C)p.omega);
    else
        collide_fluid<C>(f, m, a, (C)p.omega);
    scatter19<S, C>(dst, b.n, self, f);
}

}  // namespace lbm
