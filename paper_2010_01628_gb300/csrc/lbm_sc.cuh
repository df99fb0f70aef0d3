// lbm_sc.cuh -- device side of the Shan-Chen pseudopotential step (Sec. III.G
// of arXiv:2010.01628) shared by the single-domain kernels (lbm_sc.cu) and the
// batched persistent kernel (lbm_batch.cu): parameters, psi = 1 - exp(-rho),
// the force and macroscopic state, and the node functions of the two passes
// that the batch runs (the single-domain kernels write the same steps out).
#pragma once

#include "lbm_fluid.cuh"

namespace lbm {

struct ScArgs {
    Box box;
    double omega, G;
    double g[3];
    double rg[3];  // rho_ref g: F = rho g - rho_ref g + F_sc
    double lid[3];
};

template <typename C>
__device__ __forceinline__ C pseudopotential(C rho) {
    return (C)1 - exp(-rho);
}

// rho, F = rho g + F_sc and u = (j + F/2)/rho of a pulled node.
// NC: read-only loads of psi (it is not written during the kernel); else
// plain loads (the batched persistent kernel rewrites psi between barriers).
template <typename C, bool NC = true>
__device__ __forceinline__ Macro<C> sc_macro(const Moments<C>& m, const C* __restrict__ psi, const Box& b,
                                             const Nbr& q, int x, int y, int z, uint32_t self, const ScArgs& p) {
    Macro<C> a;
    a.rho = (C)1 + m.drho;
    const C own = NC ? psi[self] : ld_coherent(psi + self);
    C s[3];
    lattice_first_moment<C, NC>(psi, b, q, x, y, z, own, s);
    const C mg = -(C)p.G * own;
    a.Fx = (a.rho * (C)p.g[0] - (C)p.rg[0]) + mg * s[0];
    a.Fy = (a.rho * (C)p.g[1] - (C)p.rg[1]) + mg * s[1];
    a.Fz = (a.rho * (C)p.g[2] - (C)p.rg[2]) + mg * s[2];
    const C inv = recip(a.rho);
    a.ux = (m.jx + (C)0.5 * a.Fx) * inv;
    a.uy = (m.jy + (C)0.5 * a.Fy) * inv;
    a.uz = (m.jz + (C)0.5 * a.Fz) * inv;
    return a;
}

// Pass 1 at one node (batch): psi from the pulled density.
template <typename S, typename C, bool WALLS, bool NC>
__device__ __forceinline__ void sc_psi_node(const S* __restrict__ src, C* __restrict__ psi, const ScArgs& p, int x,
                                            int y, int z) {
    const Box& b = p.box;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q];
    gather19<S, C, WALLS, NC>(src, b, q, x, y, z, self, (C)p.lid[0], (C)p.lid[1], (C)p.lid[2], f);
    psi[self] = pseudopotential<C>((C)1 + moments19(f).drho);
}

// Pass 2 at one node (batch): pull, force, forced collision, mass balance, store.
template <typename S, typename C, bool WALLS, bool NC>
__device__ __forceinline__ void sc_collide_node(const S* __restrict__ src, S* __restrict__ dst,
                                                const C* __restrict__ psi, const ScArgs& p, int x, int y, int z) {
    const Box& b = p.box;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q];
    gather19<S, C, WALLS, NC>(src, b, q, x, y, z, self, (C)p.lid[0], (C)p.lid[1], (C)p.lid[2], f);
    const Moments<C> m = moments19(f);
    const Macro<C> a = sc_macro<C, NC>(m, psi, b, q, x, y, z, self, p);
    collide_fluid<C>(f, m, a, (C)p.omega);
    conserve_mass<C>(f, m.drho);
    scatter19<S, C>(dst, b.n, self, f);
}

}  // namespace lbm
