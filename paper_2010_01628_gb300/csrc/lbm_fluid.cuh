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

// One node: pull (stream + boundaries), moments, forced CM collision, store.
// NC selects the read-only load path (sources not written during the kernel).
template <typename S, typename C, bool WALLS, bool NC>
__device__ __forceinline__ void fluid_node(const S* __restrict__ src, S* __restrict__ dst, const FluidArgs& p, int x,
                                           int y, int z) {
    const Box& b = p.box;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q];
    gather19<S, C, WALLS, NC>(src, b, q, x, y, z, self, (C)p.lid[0], (C)p.lid[1], (C)p.lid[2], f);
    const Moments<C> m = moments19(f);
    const Macro<C> a = fluid_macro(m, (C)p.g[0], (C)p.g[1], (C)p.g[2]);
    collide_fluid<C>(f, m, a, (C)p.omega);
    scatter19<S, C>(dst, b.n, self, f);
}

}  // namespace lbm
