// lbm_device.cuh -- device-side building blocks of the D3Q19 central-moment
// LBM step (arXiv:2010.01628): lattice tables, storage formats, the gather
// (streaming + boundaries) and the collision in central-moment space.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// ---------------------------------------------------------------------------
// D3Q19 lattice in the paper's direction order (Sec. II.A): opposite(i) = i+9
// for i = 1..9.  Weights 1/3 (rest), 1/18 (axes), 1/36 (face diagonals).
__host__ __device__ constexpr int cx_of(int i) {
    constexpr int t[19] = {0, -1, 0, 0, -1, -1, -1, -1, 0, 0, 1, 0, 0, 1, 1, 1, 1, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int cy_of(int i) {
    constexpr int t[19] = {0, 0, -1, 0, -1, 1, 0, 0, -1, -1, 0, 1, 0, 1, -1, 0, 0, 1, 1};
    return t[i];
}
__host__ __device__ constexpr int cz_of(int i) {
    constexpr int t[19] = {0, 0, 0, -1, 0, 0, -1, 1, -1, 1, 0, 0, 1, 0, 0, 1, -1, 1, -1};
    return t[i];
}
// Runtime-index variants (for per-lane direction work).
__host__ __device__ __forceinline__ int cy_of_rt(int i) {
    return (i == 2 || i == 4 || i == 8 || i == 9 || i == 14) ? -1 : ((i == 5 || i == 11 || i == 13 || i == 17 || i == 18) ? 1 : 0);
}
__host__ __device__ __forceinline__ int cz_of_rt(int i) {
    return (i == 3 || i == 6 || i == 8 || i == 16 || i == 18) ? -1 : ((i == 7 || i == 9 || i == 12 || i == 15 || i == 17) ? 1 : 0);
}
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : (i <= 9 ? i + 9 : i - 9); }
__host__ __device__ constexpr double w_of(int i) {
    return i == 0 ? 1.0 / 3.0
                  : ((cx_of(i) * cx_of(i) + cy_of(i) * cy_of(i) + cz_of(i) * cz_of(i)) == 1 ? 1.0 / 18.0
                                                                                          : 1.0 / 36.0);
}

constexpr int Q = 19;

// Box boundary description used by every kernel.
struct Box {
    int nx, ny, nz;
    unsigned periodic;  // bit 0 x, bit 1 y, bit 2 z
    size_t n;           // nx*ny*nz (plane stride)
};

// ---------------------------------------------------------------------------
// Storage formats.  FP64/FP32 hold f - w (shift by the rest state of rho0 = 1);
// the 16-bit formats hold (f - w)/w so every direction uses the same range.
template <typename S> struct Store;
// Plain (weak, L1-cached) global loads in inline PTX, so that a const
// __restrict__ source cannot be turned into a read-only (.nc) load.
__device__ __forceinline__ double ld_coherent(const double* p) {
    double v;
    asm volatile("ld.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_coherent(const float* p) {
    float v;
    asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned short ld_coherent(const unsigned short* p) {
    unsigned short v;
    asm volatile("ld.global.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}
// load(): read-only path (ld.global.nc), valid when the source buffer is not
// written during the kernel.  load_coherent(): a plain cached load for
// persistent kernels that rewrite their sources between grid-wide barriers:
// the barrier's GPU-scope fences order it after the other CTAs' stores (the
// read-only path has no such guarantee), and it still caches in L1, which the
// neighbours' shared source values of the colour-gradient pull need.
template <> struct Store<double> {
    static constexpr bool scaled = false;
    __device__ static __forceinline__ double to_float(double v) { return v; }
    __device__ static __forceinline__ double load(const double* p) { return __ldg(p); }
    __device__ static __forceinline__ double load_coherent(const double* p) { return ld_coherent(p); }
    __device__ static __forceinline__ void store(double* p, double v) { __stcs(p, v); }
};
template <> struct Store<float> {
    static constexpr bool scaled = false;
    __device__ static __forceinline__ float to_float(float v) { return v; }
    // read-only path with the L2::256B prefetch size (a warp's 128-byte row segment also brings in its
    // neighbours'): +0.4% on the 512^3 step, up to 2% on the latency-bound multiphase and D3Q27 kernels
    __device__ static __forceinline__ float load(const float* p) {
        float v;
        asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    }
    // cached, with the same prefetch size
    __device__ static __forceinline__ float load_coherent(const float* p) {
        float v;
        asm volatile("ld.global.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    }
    __device__ static __forceinline__ void store(float* p, float v) { __stcs(p, v); }
};
template <> struct Store<__half> {
    static constexpr bool scaled = true;
    __device__ static __forceinline__ float to_float(__half v) { return __half2float(v); }
    __device__ static __forceinline__ float load(const __half* p) { return __half2float(__ldg(p)); }
    __device__ static __forceinline__ float load_coherent(const __half* p) {
        return __half2float(__ushort_as_half(ld_coherent(reinterpret_cast<const unsigned short*>(p))));
    }
    __device__ static __forceinline__ void store(__half* p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    static constexpr bool scaled = true;
    __device__ static __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __forceinline__ float load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    __device__ static __forceinline__ float load_coherent(const __nv_bfloat16* p) {
        return __uint_as_float((uint32_t)ld_coherent(reinterpret_cast<const unsigned short*>(p)) << 16);
    }
    __device__ static __forceinline__ void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// Read the shifted population f - w of direction I from storage.
template <typename S, typename C, int I, bool NC = true>
__device__ __forceinline__ C load_shifted(const S* p) {
    C v = NC ? (C)Store<S>::load(p) : (C)Store<S>::load_coherent(p);
    if (Store<S>::scaled) v *= (C)w_of(I);
    return v;
}
template <typename S, typename C, int I>
__device__ __forceinline__ void store_shifted(S* p, C v) {
    if (Store<S>::scaled) v *= (C)(1.0 / w_of(I));
    Store<S>::store(p, v);
}

// ---------------------------------------------------------------------------
// Neighbourhood of one node: wrapped neighbour coordinates along each axis and
// whether stepping off the node in that direction leaves the box through a
// wall (half-way bounce-back).
struct Nbr {
    int xm, xp, ym, yp, zm, zp;    // x-1, x+1, ... wrapped (valid only if not a wall)
    bool wxm, wxp, wym, wyp, wzm, wzp;
};

__device__ __forceinline__ Nbr make_nbr(const Box& b, int x, int y, int z) {
    Nbr q;
    const bool px = b.periodic & 1u, py = b.periodic & 2u, pz = b.periodic & 4u;
    q.xm = x == 0 ? b.nx - 1 : x - 1;
    q.xp = x == b.nx - 1 ? 0 : x + 1;
    q.ym = y == 0 ? b.ny - 1 : y - 1;
    q.yp = y == b.ny - 1 ? 0 : y + 1;
    q.zm = z == 0 ? b.nz - 1 : z - 1;
    q.zp = z == b.nz - 1 ? 0 : z + 1;
    q.wxm = !px && x == 0;
    q.wxp = !px && x == b.nx - 1;
    q.wym = !py && y == 0;
    q.wyp = !py && y == b.ny - 1;
    q.wzm = !pz && z == 0;
    q.wzp = !pz && z == b.nz - 1;
    return q;
}

// Source node of the pull x - c_i and whether it lies behind a wall.
template <int I>
__device__ __forceinline__ bool pull_source(const Box& b, const Nbr& q, int x, int y, int z, uint32_t& cell) {
    constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
    const int sx = cx == 0 ? x : (cx > 0 ? q.xm : q.xp);
    const int sy = cy == 0 ? y : (cy > 0 ? q.ym : q.yp);
    const int sz = cz == 0 ? z : (cz > 0 ? q.zm : q.zp);
    const bool wall = (cx > 0 && q.wxm) || (cx < 0 && q.wxp) || (cy > 0 && q.wym) || (cy < 0 && q.wyp) ||
                      (cz > 0 && q.wzm) || (cz < 0 && q.wzp);
    cell = ((uint32_t)sz * (uint32_t)b.ny + (uint32_t)sy) * (uint32_t)b.nx + (uint32_t)sx;
    return wall;
}

// One pulled population f_I(x) = f*_I(x - c_I) (shifted).
template <typename S, typename C, bool WALLS, int I, bool NC>
__device__ __forceinline__ C gather_one(const S* __restrict__ src, const Box& b, const Nbr& q, int x, int y, int z,
                                        uint32_t self, C lx, C ly, C lz) {
    uint32_t cell;
    const bool wall = pull_source<I>(b, q, x, y, z, cell);
    if (!WALLS) return load_shifted<S, C, I, NC>(src + (size_t)I * b.n + cell);
    // behind a wall: the node's own opposite population (same weight), chosen by
    // address rather than by a branch (+9% on the walled batch, +10% Rayleigh-Taylor)
    C v = load_shifted<S, C, I, NC>(src + (size_t)(wall ? opp_of(I) : I) * b.n + (wall ? self : cell));
    if (cy_of(I) < 0 && q.wyp)  // source beyond the +y face: the moving lid
        v += (C)(6.0 * w_of(I)) * ((C)cx_of(I) * lx + (C)cy_of(I) * ly + (C)cz_of(I) * lz);
    return v;
}

// Gather of the 19 shifted populations (Eq. streaming in pull form).  WALLS
// selects the variant with bounce-back; a pull from behind a wall reads the
// node's own post-collision population of the opposite direction, plus
// 6 w_i c_i . u_lid when the wall crossed is the moving +y lid.
template <typename S, typename C, bool WALLS, bool NC = true>
__device__ __forceinline__ void gather19(const S* __restrict__ src, const Box& b, const Nbr& q, int x, int y, int z,
                                         uint32_t self, C lx, C ly, C lz, C (&f)[Q]) {
#define LBM_G(I) f[I] = gather_one<S, C, WALLS, I, NC>(src, b, q, x, y, z, self, lx, ly, lz);
    LBM_G(0) LBM_G(1) LBM_G(2) LBM_G(3) LBM_G(4) LBM_G(5) LBM_G(6) LBM_G(7) LBM_G(8) LBM_G(9) LBM_G(10)
    LBM_G(11) LBM_G(12) LBM_G(13) LBM_G(14) LBM_G(15) LBM_G(16) LBM_G(17) LBM_G(18)
#undef LBM_G
}

// Value of a node field v at x + c_I; a neighbour behind a wall contributes
// the node's own value `own`.  NC: read-only path (the field is not written
// during the kernel); else a plain load (persistent kernels that rewrite the
// field between grid-wide barriers; see Store::load_coherent).
template <typename C, int I, bool NC = true>
__device__ __forceinline__ C field_nbr(const C* __restrict__ v, const Box& b, const Nbr& q, int x, int y, int z,
                                       C own) {
    constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
    const int sx = cx == 0 ? x : (cx > 0 ? q.xp : q.xm);
    const int sy = cy == 0 ? y : (cy > 0 ? q.yp : q.ym);
    const int sz = cz == 0 ? z : (cz > 0 ? q.zp : q.zm);
    const bool wall = (cx > 0 && q.wxp) || (cx < 0 && q.wxm) || (cy > 0 && q.wyp) || (cy < 0 && q.wym) ||
                      (cz > 0 && q.wzp) || (cz < 0 && q.wzm);
    if (wall) return own;
    const C* a = v + ((uint32_t)sz * (uint32_t)b.ny + (uint32_t)sy) * (uint32_t)b.nx + (uint32_t)sx;
    return NC ? __ldg(a) : ld_coherent(a);
}

// s = sum_i w_i c_i v(x + c_i) over the 18 moving directions: the lattice
// first moment of a node field (times 1/c_s^2 the isotropic gradient of the
// colour-gradient model; times -G psi(x) the Shan-Chen force).
template <typename C, bool NC = true>
__device__ __forceinline__ void lattice_first_moment(const C* __restrict__ v, const Box& b, const Nbr& q, int x,
                                                     int y, int z, C own, C (&s)[3]) {
    C gx = (C)0, gy = (C)0, gz = (C)0;
#define LBM_FM(I)                                                           \
    {                                                                       \
        const C t = field_nbr<C, I, NC>(v, b, q, x, y, z, own) * (C)w_of(I); \
        if (cx_of(I)) gx += (C)cx_of(I) * t;                                \
        if (cy_of(I)) gy += (C)cy_of(I) * t;                                \
        if (cz_of(I)) gz += (C)cz_of(I) * t;                                \
    }
    LBM_FM(1) LBM_FM(2) LBM_FM(3) LBM_FM(4) LBM_FM(5) LBM_FM(6) LBM_FM(7) LBM_FM(8) LBM_FM(9) LBM_FM(10)
    LBM_FM(11) LBM_FM(12) LBM_FM(13) LBM_FM(14) LBM_FM(15) LBM_FM(16) LBM_FM(17) LBM_FM(18)
#undef LBM_FM
    s[0] = gx;
    s[1] = gy;
    s[2] = gz;
}

template <typename S, typename C>
__device__ __forceinline__ void scatter19(S* __restrict__ dst, size_t n, uint32_t self, const C (&f)[Q]) {
#define LBM_STORE(I) store_shifted<S, C, I>(dst + (size_t)I * n + self, f[I]);
    LBM_STORE(0) LBM_STORE(1) LBM_STORE(2) LBM_STORE(3) LBM_STORE(4) LBM_STORE(5) LBM_STORE(6) LBM_STORE(7)
    LBM_STORE(8) LBM_STORE(9) LBM_STORE(10) LBM_STORE(11) LBM_STORE(12) LBM_STORE(13) LBM_STORE(14)
    LBM_STORE(15) LBM_STORE(16) LBM_STORE(17) LBM_STORE(18)
#undef LBM_STORE
}

// ---------------------------------------------------------------------------
// Raw moments of the shifted populations: d = sum (f - w) = rho - 1, the
// momentum j = sum f c, and the shifted second moments (the w parts of
// sum f c_a c_b cancel in every combination used below).
template <typename C>
struct Moments {
    C drho, jx, jy, jz;
    C pxx_m_pyy, pyy_m_pzz, pxy, pxz, pyz;
    C moving;  // sum of the 18 moving populations; drho = moving + f_0
};

template <typename C>
__device__ __forceinline__ Moments<C> moments19(const C (&f)[Q]) {
    Moments<C> m;
    const C sx_p = f[10] + f[13] + f[14] + f[15] + f[16];  // c_x = +1
    const C sx_m = f[1] + f[4] + f[5] + f[6] + f[7];       // c_x = -1
    const C sy_p = f[5] + f[11] + f[13] + f[17] + f[18];
    const C sy_m = f[2] + f[4] + f[8] + f[9] + f[14];
    const C sz_p = f[7] + f[9] + f[12] + f[15] + f[17];
    const C sz_m = f[3] + f[6] + f[8] + f[16] + f[18];
    m.jx = sx_p - sx_m;
    m.jy = sy_p - sy_m;
    m.jz = sz_p - sz_m;
    // sum_i f c_a^2: directions with c_a != 0 are exactly those counted above
    const C pxx = sx_p + sx_m, pyy = sy_p + sy_m, pzz = sz_p + sz_m;
    // c_x = 0 directions: 0, 2, 3, 8, 9, 11, 12, 17, 18; the rest population
    // is added last (conserve_mass relies on this order)
    m.moving = pxx + (f[2] + f[11]) + (f[3] + f[12]) + (f[8] + f[17]) + (f[9] + f[18]);
    m.drho = m.moving + f[0];
    m.pxx_m_pyy = pxx - pyy;
    m.pyy_m_pzz = pyy - pzz;
    m.pxy = (f[4] + f[13]) - (f[5] + f[14]);
    m.pxz = (f[6] + f[15]) - (f[7] + f[16]);
    m.pyz = (f[8] + f[17]) - (f[9] + f[18]);
    return m;
}

// moments19 from the stored values of the 16-bit formats, q_i = (f_i - w_i)/w_i,
// without scaling each population first: the sums run over
// 36 (f_i - w_i) = 12 q_0, 2 q_i (axes), q_i (diagonals), and the nine moments
// the collision uses are scaled by 1/36 at the end (`moving` is left x36).
template <typename C>
__device__ __forceinline__ Moments<C> moments19_q(const C (&q)[Q]) {
    Moments<C> m;
    const C two = (C)2, k = (C)(1.0 / 36.0);
    const C sx_p = two * q[10] + q[13] + q[14] + q[15] + q[16];
    const C sx_m = two * q[1] + q[4] + q[5] + q[6] + q[7];
    const C sy_p = two * q[11] + q[5] + q[13] + q[17] + q[18];
    const C sy_m = two * q[2] + q[4] + q[8] + q[9] + q[14];
    const C sz_p = two * q[12] + q[7] + q[9] + q[15] + q[17];
    const C sz_m = two * q[3] + q[6] + q[8] + q[16] + q[18];
    m.jx = (sx_p - sx_m) * k;
    m.jy = (sy_p - sy_m) * k;
    m.jz = (sz_p - sz_m) * k;
    const C pxx = sx_p + sx_m, pyy = sy_p + sy_m, pzz = sz_p + sz_m;
    m.moving = pxx + two * ((q[2] + q[11]) + (q[3] + q[12])) + ((q[8] + q[17]) + (q[9] + q[18]));
    m.drho = ((C)12 * q[0] + m.moving) * k;
    m.pxx_m_pyy = (pxx - pyy) * k;
    m.pyy_m_pzz = (pyy - pzz) * k;
    m.pxy = ((q[4] + q[13]) - (q[5] + q[14])) * k;
    m.pxz = ((q[6] + q[15]) - (q[7] + q[16])) * k;
    m.pyz = ((q[8] + q[17]) - (q[9] + q[18])) * k;
    return m;
}

// Sets the rest population so that the 19 values sum to drho in the order of
// the next step's density sum (moving directions first, f_0 last).  The
// rounding error of f_0 = drho - S is at most half an ulp of f_0, so whenever
// |f_0| <= |drho| the next sum S + f_0 rounds back to drho itself (barring an
// exact tie).  A uniform region (both phases of a multiphase run) then keeps
// its mass exactly in FP32 instead of repeating the same rounding error at
// every node and step.  Values are the shifted f - w.
template <typename C>
__device__ __forceinline__ void conserve_mass(C (&f)[Q], C drho) {
    f[0] = drho - moments19(f).moving;
}

// f = M^-1 r (App. C, Eq. pdfQ19): populations from the 19 raw moments.
// Each axis pair shares its common part (f_-/+ = E +- D) and each group of four
// diagonal directions its sums and differences (f4, f5, f13, f14 =
// (P +- D)/4, (P' +- S)/4 with P = r16 - r11, P' = r16 + r11, D = r7 - r10,
// S = r7 + r10): fewer operations for the FP64 pipe, which bounds the FP64
// step, and for the issue-bound colour-gradient collision.
template <typename C>
__device__ __forceinline__ void raw_to_populations(const C (&r)[Q], C (&f)[Q]) {
    const C half = (C)0.5, mhalf = (C)-0.5, quarter = (C)0.25, mquarter = (C)-0.25, sixth = (C)(1.0 / 6.0);
    const C ax = (r[4] + (C)2 * r[5] + r[6]) * sixth;
    const C ay = (r[4] - r[5] + r[6]) * sixth;
    const C az = (r[4] - r[5] - (C)2 * r[6]) * sixth;
    const C s1617 = r[16] + r[17], s1618 = r[16] + r[18], s1718 = r[17] + r[18];
    f[0] = r[0] - r[4] + r[16] + s1718;
    {
        const C e = s1617 * mhalf + ax, d = (r[11] + r[13] - r[1]) * half;
        f[1] = e + d;
        f[10] = e - d;
    }
    {
        const C e = s1618 * mhalf + ay, d = (r[10] + r[15] - r[2]) * half;
        f[2] = e + d;
        f[11] = e - d;
    }
    {
        const C e = s1718 * mhalf + az, d = (r[12] + r[14] - r[3]) * half;
        f[3] = e + d;
        f[12] = e - d;
    }
    {
        const C pm = (r[16] - r[11]) * quarter, pp = (r[16] + r[11]) * quarter, dm = r[7] - r[10], dp = r[7] + r[10];
        f[4] = dm * quarter + pm;
        f[5] = dm * mquarter + pm;
        f[13] = dp * quarter + pp;
        f[14] = dp * mquarter + pp;
    }
    {
        const C pm = (r[17] - r[13]) * quarter, pp = (r[17] + r[13]) * quarter, dm = r[8] - r[12], dp = r[8] + r[12];
        f[6] = dm * quarter + pm;
        f[7] = dm * mquarter + pm;
        f[15] = dp * quarter + pp;
        f[16] = dp * mquarter + pp;
    }
    {
        const C pm = (r[18] - r[15]) * quarter, pp = (r[18] + r[15]) * quarter, dm = r[9] - r[14], dp = r[9] + r[14];
        f[8] = dm * quarter + pm;
        f[9] = dm * mquarter + pm;
        f[17] = dp * quarter + pp;
        f[18] = dp * mquarter + pp;
    }
}

// raw_to_populations with the result in the 16-bit formats' units,
// q_i = (f_i - w_i)/w_i = 3 f_0, 18 f_i (axes), 36 f_i (diagonals): the 1/w_i
// scaling rides on the constants of M^-1 instead of costing a multiply per
// population.  Each group of four diagonal directions shares its sums and
// differences (e.g. q4, q5, q13, q14 = 9 (P +- D), 9 (P' +- S) with
// P = r16 - r11, P' = r16 + r11, D = r7 - r10, S = r7 + r10), and each axis
// pair its common part, which the packed two-node collision of the 16-bit
// kernels, bound by FP32-pipe operations, needs.
template <typename C>
__device__ __forceinline__ void raw_to_populations_q(const C (&r)[Q], C (&q)[Q]) {
    const C nine = (C)9, mnine = (C)-9, three = (C)3;
    const C ax = (r[4] + (C)2 * r[5] + r[6]) * three;
    const C ay = (r[4] - r[5] + r[6]) * three;
    const C az = (r[4] - r[5] - (C)2 * r[6]) * three;
    const C s1617 = r[16] + r[17], s1618 = r[16] + r[18], s1718 = r[17] + r[18];
    q[0] = (r[0] - r[4] + r[16] + s1718) * three;
    // axes: q_+ = E - D, q_- = E + D with E = a - 9 s, D = 9 (r_b - r_1)
    {
        const C e = s1617 * mnine + ax, d = (r[11] + r[13] - r[1]) * nine;
        q[1] = e + d;
        q[10] = e - d;
    }
    {
        const C e = s1618 * mnine + ay, d = (r[10] + r[15] - r[2]) * nine;
        q[2] = e + d;
        q[11] = e - d;
    }
    {
        const C e = s1718 * mnine + az, d = (r[12] + r[14] - r[3]) * nine;
        q[3] = e + d;
        q[12] = e - d;
    }
    // face diagonals, four per plane
    {
        const C pm = (r[16] - r[11]) * nine, pp = (r[16] + r[11]) * nine, dm = r[7] - r[10], dp = r[7] + r[10];
        q[4] = dm * nine + pm;
        q[5] = dm * mnine + pm;
        q[13] = dp * nine + pp;
        q[14] = dp * mnine + pp;
    }
    {
        const C pm = (r[17] - r[13]) * nine, pp = (r[17] + r[13]) * nine, dm = r[8] - r[12], dp = r[8] + r[12];
        q[6] = dm * nine + pm;
        q[7] = dm * mnine + pm;
        q[15] = dp * nine + pp;
        q[16] = dp * mnine + pp;
    }
    {
        const C pm = (r[18] - r[15]) * nine, pp = (r[18] + r[15]) * nine, dm = r[9] - r[14], dp = r[9] + r[14];
        q[8] = dm * nine + pm;
        q[9] = dm * mnine + pm;
        q[17] = dp * nine + pp;
        q[18] = dp * mnine + pp;
    }
}

// ---------------------------------------------------------------------------
// Back-transform of App. C in two steps, r* = N^-1 k* (Eq. rawQ19) then
// f* = M^-1 r* (Eq. pdfQ19), for a post-collision CM vector with
//   k1..3 = h (= F/2), k4 (enters the products with u), k5..9 = kd[0..4],
//   k10..15 = t[0..5], and the "standalone" parts r0c (of r0), k4c (of r4),
//   k16c..18c (of r16..18).
// With r0c = rho - 1, k4c = k4 - 1 and k16c = k16 - 1/9 the result is
// f* - w directly (M^-1 maps (1,0,0,0,1,0..0,1/9,1/9,1/9) to w), so shifted
// storage loses no digits to the O(1) rest state.  The c_s^2 factors on the
// k5/k6 terms of r16..18 follow from the expansion c = cbar + u.
// QOUT: the result in the 16-bit units q = (f* - w)/w (raw_to_populations_q).
// px, py, pz: the post-collision momentum r1..3* = rho u + h, passed in by the
// caller as sum f c + F (the same value, without the division by rho and the
// product with it: in FP32 that round trip biased the momentum of a uniformly
// accelerated flow by 1e-5 of itself over 1000 steps).
template <typename C, bool QOUT = false>
__device__ __forceinline__ void back_transform(C rho, C ux, C uy, C uz, C hx, C hy, C hz, C px, C py, C pz, C k4,
                                               C r0c, C k4c, const C (&kd)[5], const C (&t)[6], C k16c, C k17c,
                                               C k18c, C (&f)[Q]) {
    const C third = (C)(1.0 / 3.0);
    const C x2 = ux * ux, y2 = uy * uy, z2 = uz * uz;
    const C k5 = kd[0], k6 = kd[1], k7 = kd[2], k8 = kd[3], k9 = kd[4];
    // sum f cbar_x^2 etc. expressed through k4, k5, k6 (times c_s^2 = 1/3)
    const C Xs = (k4 + (C)2 * k5 + k6) * third;  // sum f cbar_x^2
    const C Ys = (k4 - k5 + k6) * third;         // sum f cbar_y^2
    const C Zs = (k4 - k5 - (C)2 * k6) * third;  // sum f cbar_z^2

    C r[Q];
    r[0] = r0c;
    r[1] = px;
    r[2] = py;
    r[3] = pz;
    r[4] = rho * (x2 + y2 + z2) + (C)2 * (ux * hx + uy * hy + uz * hz) + k4c;
    r[5] = rho * (x2 - y2) + (C)2 * (ux * hx - uy * hy) + k5;
    r[6] = rho * (y2 - z2) + (C)2 * (uy * hy - uz * hz) + k6;
    r[7] = rho * ux * uy + uy * hx + ux * hy + k7;
    r[8] = rho * ux * uz + uz * hx + ux * hz + k8;
    r[9] = rho * uy * uz + uz * hy + uy * hz + k9;
    // third order: sum f c_a^2 c_b = k(a^2 b) + u_b Xa + 2 u_a k(ab) + 2 u_a u_b h_a + u_a^2 h_b + rho u_a^2 u_b,
    // grouped as u_a^2 (rho u_b + h_b) + u_b (2 u_a h_a + Xa) + 2 u_a k(ab) + k(a^2 b)
    const C Ax = (C)2 * ux * hx + Xs, Ay = (C)2 * uy * hy + Ys, Az = (C)2 * uz * hz + Zs;
    const C tx = (C)2 * ux, ty = (C)2 * uy, tz = (C)2 * uz;
    r[10] = x2 * r[2] + uy * Ax + tx * k7 + t[0];
    r[11] = y2 * r[1] + ux * Ay + ty * k7 + t[1];
    r[12] = x2 * r[3] + uz * Ax + tx * k8 + t[2];
    r[13] = z2 * r[1] + ux * Az + tz * k8 + t[3];
    r[14] = y2 * r[3] + uz * Ay + ty * k9 + t[4];
    r[15] = z2 * r[2] + uy * Az + tz * k9 + t[5];
    // fourth order: sum f c_a^2 c_b^2 = u_b^2 (rho u_a^2 + A_a) + u_a^2 A_b + 2 u_a (2 u_b k(ab) + k(a b^2))
    //                                   + 2 u_b k(a^2 b) + k(a^2 b^2)
    const C rx2 = rho * x2, ry2 = rho * y2;
    r[16] = y2 * (rx2 + Ax) + x2 * Ay + tx * (ty * k7 + t[1]) + ty * t[0] + k16c;
    r[17] = z2 * (rx2 + Ax) + x2 * Az + tx * (tz * k8 + t[3]) + tz * t[2] + k17c;
    r[18] = z2 * (ry2 + Ay) + y2 * Az + ty * (tz * k9 + t[5]) + tz * t[4] + k18c;

    if (QOUT)
        raw_to_populations_q<C>(r, f);
    else
        raw_to_populations<C>(r, f);
}

// 1/x: correctly rounded reciprocal (the FP32 division would add a slow path).
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Macroscopic state of a gathered node: rho, F, u = (sum f c + F/2)/rho.
template <typename C>
struct Macro {
    C rho, ux, uy, uz, Fx, Fy, Fz;
};

// Single-phase forced CM collision (Sec. II.B, list after Eq. eq:posColl0),
// in shifted variables: f holds f - w on entry and f* - w on exit (QOUT: the
// 16-bit units (f* - w)/w on exit).
template <typename C, bool QOUT = false>
__device__ __forceinline__ void collide_fluid(C (&f)[Q], const Moments<C>& m, const Macro<C>& a, C omega) {
    const C rho = a.rho, ux = a.ux, uy = a.uy, uz = a.uz;
    const C hx = (C)0.5 * a.Fx, hy = (C)0.5 * a.Fy, hz = (C)0.5 * a.Fz;
    const C om1 = (C)1 - omega;
    // pre-collision central second moments (Eq. pre_collision_central_moments)
    // from raw moments: sum f cbar_a cbar_b = P_ab - rho u_a u_b + (u_a F_b + u_b F_a)/2
    C kd[5];
    kd[0] = om1 * (m.pxx_m_pyy - rho * (ux * ux - uy * uy) + (C)2 * (ux * hx - uy * hy));
    kd[1] = om1 * (m.pyy_m_pzz - rho * (uy * uy - uz * uz) + (C)2 * (uy * hy - uz * hz));
    kd[2] = om1 * (m.pxy - rho * ux * uy + ux * hy + uy * hx);
    kd[3] = om1 * (m.pxz - rho * ux * uz + ux * hz + uz * hx);
    kd[4] = om1 * (m.pyz - rho * uy * uz + uy * hz + uz * hy);
    const C third = (C)(1.0 / 3.0);
    // k10..15* = c_s^2 F/2 in the order (Fy, Fx, Fz, Fx, Fz, Fy)
    const C t[6] = {hy * third, hx * third, hz * third, hx * third, hz * third, hy * third};
    const C drho = m.drho;
    const C k16c = drho * (C)(1.0 / 9.0);
    back_transform<C, QOUT>(rho, ux, uy, uz, hx, hy, hz, m.jx + a.Fx, m.jy + a.Fy, m.jz + a.Fz, rho, drho, drho, kd,
                            t, k16c, k16c, k16c, f);
}

// Raw-moment variant (App. C, N = I, T = M): r* = k* from the printed list, in
// the shifted variables (the rest state's raw moments r0 = 1, r4 = 3 c_s^2 = 1,
// r16..18 = c_s^4 = 1/9 subtracted exactly), then f* = M^-1 r*.
//   r1..3* = rho u + F/2; r4* = rho (3 c_s^2 + |u|^2);
//   r5..9* = (1 - omega) r5..9 + omega rho (u u)_5..9;
//   r10..15* = c_s^2 F/2 + rho u_b (u_a^2 + c_s^2); r16..18* = rho (u_a^2 + c_s^2)(u_b^2 + c_s^2).
template <typename C>
__device__ __forceinline__ void collide_fluid_rm(C (&f)[Q], const Moments<C>& m, const Macro<C>& a, C omega) {
    const C rho = a.rho, ux = a.ux, uy = a.uy, uz = a.uz;
    const C hx = (C)0.5 * a.Fx, hy = (C)0.5 * a.Fy, hz = (C)0.5 * a.Fz;
    const C x2 = ux * ux, y2 = uy * uy, z2 = uz * uz;
    const C om1 = (C)1 - omega, third = (C)(1.0 / 3.0), ninth = (C)(1.0 / 9.0);
    const C drho = m.drho;
    C r[Q];
    r[0] = drho;
    r[1] = rho * ux + hx;
    r[2] = rho * uy + hy;
    r[3] = rho * uz + hz;
    r[4] = drho + rho * (x2 + y2 + z2);
    r[5] = om1 * m.pxx_m_pyy + omega * rho * (x2 - y2);
    r[6] = om1 * m.pyy_m_pzz + omega * rho * (y2 - z2);
    r[7] = om1 * m.pxy + omega * rho * ux * uy;
    r[8] = om1 * m.pxz + omega * rho * ux * uz;
    r[9] = om1 * m.pyz + omega * rho * uy * uz;
    const C ax = x2 + third, ay = y2 + third, az = z2 + third;
    const C rux = rho * ux, ruy = rho * uy, ruz = rho * uz;
    r[10] = hy * third + ruy * ax;
    r[11] = hx * third + rux * ay;
    r[12] = hz * third + ruz * ax;
    r[13] = hx * third + rux * az;
    r[14] = hz * third + ruz * ay;
    r[15] = hy * third + ruy * az;
    r[16] = rho * (x2 * y2 + (x2 + y2) * third) + drho * ninth;
    r[17] = rho * (x2 * z2 + (x2 + z2) * third) + drho * ninth;
    r[18] = rho * (y2 * z2 + (y2 + z2) * third) + drho * ninth;
    raw_to_populations<C>(r, f);
}

// Equilibrium of (rho, u) in shifted form: the back-transform of k_eq.
template <typename C>
__device__ __forceinline__ void equilibrium_shifted(C rho, C drho, C ux, C uy, C uz, C (&f)[Q]) {
    const C z = (C)0;
    const C kd[5] = {z, z, z, z, z};
    const C t[6] = {z, z, z, z, z, z};
    const C k16c = drho * (C)(1.0 / 9.0);
    back_transform<C>(rho, ux, uy, uz, z, z, z, rho * ux, rho * uy, rho * uz, rho, drho, drho, kd, t, k16c, k16c,
                      k16c, f);
}

// ---------------------------------------------------------------------------
// TMA bulk copies and mbarriers (inline PTX, sm_90+ forms valid on sm_103a).
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// 1D bulk copy global -> shared, completion counted on `bar` (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for phase `parity` of `bar`; false if the deadline passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

}  // namespace lbm
