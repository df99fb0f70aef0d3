// lbm_fluid.cu -- single-phase D3Q19 central-moment step (Sec. II of
// arXiv:2010.01628) with a constant body force, in four storage precisions.
//
// One thread per node, a block along x.  Each step is one fused pass:
// pull the 19 post-collision populations of the neighbours (periodic wrap or
// half-way bounce-back), form rho and u = (sum f c + F/2)/rho, relax the five
// deviatoric central second moments by (1 - omega), set every other central
// moment to its forced equilibrium value, rebuild f* with the two-step
// transform of App. C and store it, coalesced, to the other buffer.
#include "lbm_fluid.cuh"
#include "lbm_pack2.cuh"
#include "lbm_internal.h"
#include "lbm_reduce.cuh"

namespace lbm {

template <typename S, typename C, bool WALLS, bool RM = false>
__global__ void __launch_bounds__(256) fluid_step_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                         FluidArgs p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.box.nx) return;
    fluid_node<S, C, WALLS, true, RM>(src, dst, p, x, blockIdx.y, blockIdx.z);
}

// Channels (x and z periodic, walls on y, ny >= 3) step in two launches: the
// interior rows 1 .. ny-2 never pull through a wall and run the periodic node
// code (40 registers instead of 48); a small launch then updates the two wall
// rows with bounce-back or regularized walls.
template <typename S, typename C>
__global__ void __launch_bounds__(256) fluid_step_interior_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                                  FluidArgs p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.box.nx) return;
    fluid_node<S, C, false, true>(src, dst, p, x, blockIdx.y + 1, blockIdx.z);
}

// The wall rows y = 0 (blockIdx.y = 0) and y = ny - 1 (blockIdx.y = 1) of a
// channel.  REG: regularized on-node walls; else half-way bounce-back with the lid.
template <typename S, typename C, bool REG>
__global__ void __launch_bounds__(256) fluid_step_wallrows_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                                  FluidArgs p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const Box& b = p.box;
    const int y = blockIdx.y == 0 ? 0 : b.ny - 1, z = blockIdx.z;
    if (x >= b.nx) return;
    if (!REG) {
        fluid_node<S, C, true, true>(src, dst, p, x, y, z);
        return;
    }
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C f[Q];
    gather_regularized<S, C>(src, p, q, x, y, z, self, f);
    const Moments<C> m = moments19(f);
    const Macro<C> a = fluid_macro(m, (C)p.g[0], (C)p.g[1], (C)p.g[2]);
    collide_fluid<C>(f, m, a, (C)p.omega);
    scatter19<S, C>(dst, b.n, self, f);
}

// ---------------------------------------------------------------------------
// Read-only loads that ask L2 to fetch the surrounding 256-byte block from DRAM
// (ld.global.nc with the L2::256B prefetch size): a warp's 128-byte (x-pairs)
// or 64-byte (z-pairs) row segment also brings in its neighbouring warps'
// segments, which then wait for L2 instead of DRAM.  About 1% on the
// latency-bound 16-bit kernels.
__device__ __forceinline__ uint32_t ldg_l2pf(const uint32_t* p) {
    uint32_t v;
    asm("ld.global.nc.L2::256B.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
template <typename S>
__device__ __forceinline__ float ldg_l2pf(const S* p) {
    unsigned short v;
    asm("ld.global.nc.L2::256B.u16 %0, [%1];" : "=h"(v) : "l"(p));
    S h;
    *reinterpret_cast<unsigned short*>(&h) = v;
    return Store<S>::to_float(h);
}

// ---------------------------------------------------------------------------
// 16-bit storage, two adjacent x-cells per thread.  A thread owns the 32-bit
// word holding cells (x0, x0+1), x0 even, of every plane: all loads and stores
// are aligned 4-byte accesses (128 B per warp per plane).  Directions with
// c_x = +1 need (x0-1, x0): the high half of the previous word, taken from
// lane-1 by a shuffle (lane 0 and the row start load it); c_x = -1 needs
// (x0+1, x0+2): the low half of the next word from lane+1 (lane 31 and the row
// end load it).  Requires nx even.
template <typename S>
struct Pair16;
template <>
struct Pair16<__half> {
    __device__ static __forceinline__ float lo(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
    __device__ static __forceinline__ float hi(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
    // one conversion instruction rounds and packs both lanes (x low, y high)
    __device__ static __forceinline__ uint32_t pack(float2 v) {
        const __half2 h = __floats2half2_rn(v.x, v.y);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
};
template <>
struct Pair16<__nv_bfloat16> {
    __device__ static __forceinline__ float lo(uint32_t w) { return __uint_as_float(w << 16); }
    __device__ static __forceinline__ float hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
    __device__ static __forceinline__ uint32_t pack(float2 v) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
};

struct PairCtx {
    int x0, lane;
    bool active;
    uint32_t self_w;  // word index of the thread's cells within a plane
    uint32_t plane_w; // words per plane
};

// The pull of direction I for the thread's two cells, in two phases so that
// all 19 directions' loads are in flight before the first is consumed.
// Phase 1: the thread's own word of the source row and, for a lane at the
// warp's or the row's edge, the neighbouring word no neighbour lane holds.
template <bool WALLS, int I>
__device__ __forceinline__ void pair_words(const uint32_t* __restrict__ src, const Box& b, const Nbr& q,
                                           const PairCtx& t, int y, int z, uint32_t& wv, uint32_t& ev) {
    constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
    const int sy = cy == 0 ? y : (cy > 0 ? q.ym : q.yp);
    const int sz = cz == 0 ? z : (cz > 0 ? q.zm : q.zp);
    const bool row_wall = WALLS && ((cy > 0 && q.wym) || (cy < 0 && q.wyp) || (cz > 0 && q.wzm) || (cz < 0 && q.wzp));
    const uint32_t* P = src + (size_t)I * t.plane_w + ((((uint32_t)sz * (uint32_t)b.ny + (uint32_t)sy) * (uint32_t)b.nx) >> 1);
    const uint32_t own = (uint32_t)t.x0 >> 1;
    const bool ld = t.active && !row_wall;
    wv = ld ? ldg_l2pf(P + own) : 0u;
    ev = 0u;
    if (cx > 0 && ld && (t.lane == 0 || t.x0 == 0)) ev = __ldg(P + (t.x0 == 0 ? (uint32_t)(b.nx - 2) >> 1 : own - 1));
    if (cx < 0 && ld && (t.lane == 31 || t.x0 + 2 >= b.nx)) ev = __ldg(P + (t.x0 + 2 >= b.nx ? 0u : own + 1));
}

// Phase 2: the two cells' values of direction I, in the stored units
// q = (f - w)/w, from the words (x-shifted directions take the neighbouring
// half by a shuffle), with half-way bounce-back replacements.  Every lane of
// the warp executes the shuffles (inactive lanes past the row end carry zeros).
template <typename S, bool WALLS, int I>
__device__ __forceinline__ P2 pair_combine(const uint32_t* __restrict__ src, const Box& b, const Nbr& q,
                                           const PairCtx& t, uint32_t wv, uint32_t ev, float lx, float ly,
                                           float lz) {
    constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
    uint32_t val = wv;
    if (cx > 0) {  // cells need elements (x0 - 1, x0)
        uint32_t pv = __shfl_up_sync(0xffffffffu, wv, 1);
        if (t.lane == 0 || t.x0 == 0) pv = ev;
        val = __byte_perm(pv, wv, 0x5432);
    } else if (cx < 0) {  // cells need elements (x0 + 1, x0 + 2)
        uint32_t nv = __shfl_down_sync(0xffffffffu, wv, 1);
        if (t.lane == 31 || t.x0 + 2 >= b.nx) nv = ev;
        val = __byte_perm(wv, nv, 0x5432);
    }
    P2 f = P2(Pair16<S>::lo(val), Pair16<S>::hi(val));
    if (WALLS) {
        // half-way bounce-back: the node's own post-collision population of the
        // opposite direction (+ the moving-lid term when the +y face is crossed)
        const bool row_wall = (cy > 0 && q.wym) || (cy < 0 && q.wyp) || (cz > 0 && q.wzm) || (cz < 0 && q.wzp);
        const bool wall_a = row_wall || (cx > 0 && q.wxm);
        const bool wall_b = row_wall || (cx < 0 && t.x0 + 1 == b.nx - 1 && !(b.periodic & 1u));
        if (wall_a || wall_b) {
            const uint32_t ov = t.active ? __ldg(src + (size_t)opp_of(I) * t.plane_w + t.self_w) : 0u;
            // the lid term 6 w c.u_lid is 6 c.u_lid in units of w
            const float lid = (cy < 0 && q.wyp) ? 6.f * ((float)cx * lx + (float)cy * ly + (float)cz * lz) : 0.f;
            if (wall_a) f.v.x = Pair16<S>::lo(ov) + lid;
            if (wall_b) f.v.y = Pair16<S>::hi(ov) + lid;
        }
    }
    return f;
}

// Phase 1 for all 19 directions of plane z (row y).
template <bool WALLS>
__device__ __forceinline__ void pair_words_all(const uint32_t* __restrict__ src, const Box& b, const Nbr& q,
                                               const PairCtx& t, int y, int z, uint32_t (&wv)[Q], uint32_t (&ev)[Q]) {
#define LBM_PW(I) pair_words<WALLS, I>(src, b, q, t, y, z, wv[I], ev[I]);
    LBM_PW(0) LBM_PW(1) LBM_PW(2) LBM_PW(3) LBM_PW(4) LBM_PW(5) LBM_PW(6) LBM_PW(7) LBM_PW(8) LBM_PW(9)
    LBM_PW(10) LBM_PW(11) LBM_PW(12) LBM_PW(13) LBM_PW(14) LBM_PW(15) LBM_PW(16) LBM_PW(17) LBM_PW(18)
#undef LBM_PW
}

// Phase 2 and the rest of the update of the thread's two cells: both through
// one packed collision in the stored units q = (f - w)/w, then one 32-bit
// store per direction.  All lanes take part in the shuffles.
template <typename S, bool WALLS>
__device__ __forceinline__ void pair_relax_store(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                                                 const FluidArgs& p, const Nbr& q, const PairCtx& t,
                                                 const uint32_t (&wv)[Q], const uint32_t (&ev)[Q], float lx,
                                                 float ly, float lz) {
    const Box& b = p.box;
    P2 f[Q];
#define LBM_GP(I) f[I] = pair_combine<S, WALLS, I>(src, b, q, t, wv[I], ev[I], lx, ly, lz);
    LBM_GP(0) LBM_GP(1) LBM_GP(2) LBM_GP(3) LBM_GP(4) LBM_GP(5) LBM_GP(6) LBM_GP(7) LBM_GP(8) LBM_GP(9)
    LBM_GP(10) LBM_GP(11) LBM_GP(12) LBM_GP(13) LBM_GP(14) LBM_GP(15) LBM_GP(16) LBM_GP(17) LBM_GP(18)
#undef LBM_GP
    if (!t.active) return;
    const Moments<P2> m = moments19_q(f);
    const Macro<P2> a = fluid_macro(m, P2((float)p.g[0]), P2((float)p.g[1]), P2((float)p.g[2]));
    collide_fluid<P2, true>(f, m, a, P2((float)p.omega));
#define LBM_SP(I) __stcs(dst + (size_t)I * t.plane_w + t.self_w, Pair16<S>::pack(f[I].v));
    LBM_SP(0) LBM_SP(1) LBM_SP(2) LBM_SP(3) LBM_SP(4) LBM_SP(5) LBM_SP(6) LBM_SP(7) LBM_SP(8) LBM_SP(9)
    LBM_SP(10) LBM_SP(11) LBM_SP(12) LBM_SP(13) LBM_SP(14) LBM_SP(15) LBM_SP(16) LBM_SP(17) LBM_SP(18)
#undef LBM_SP
}

__device__ __forceinline__ PairCtx pair_ctx(const Box& b) {
    PairCtx t;
    t.x0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    t.lane = threadIdx.x & 31;
    t.active = t.x0 < b.nx;
    t.plane_w = (uint32_t)(b.n >> 1);
    return t;
}
__device__ __forceinline__ uint32_t pair_self(const Box& b, const PairCtx& t, int y, int z) {
    return ((((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx) >> 1) + ((uint32_t)t.x0 >> 1);
}

template <typename S, bool WALLS>
__global__ void __launch_bounds__(256) fluid_step_pair_kernel(const S* __restrict__ src_, S* __restrict__ dst_,
                                                              FluidArgs p) {
    const Box& b = p.box;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(src_);
    uint32_t* dst = reinterpret_cast<uint32_t*>(dst_);
    const int y = blockIdx.y, z = blockIdx.z;
    PairCtx t = pair_ctx(b);
    t.self_w = pair_self(b, t, y, z);
    // x-neighbour flags of cell x0 (left wall) and of the row; the right wall
    // of cell x0+1 is tested in pair_combine
    const Nbr q = make_nbr(b, t.active ? t.x0 : 0, y, z);
    uint32_t wv[Q], ev[Q];
    pair_words_all<WALLS>(src, b, q, t, y, z, wv, ev);
    pair_relax_store<S, WALLS>(src, dst, p, q, t, wv, ev, (float)p.lid[0], (float)p.lid[1], (float)p.lid[2]);
}

// ---------------------------------------------------------------------------
// 16-bit storage, two nodes per thread stacked in z: (x, y, z0) and
// (x, y, z0 + 1), z0 even (for odd nz the last thread updates z0 alone).  Every
// pull is a plain 2-byte load of the stored q = (f - w)/w; one packed collision
// relaxes both nodes in those units (the w scalings ride on the moment sums and
// on M^-1) before the two stores.
template <typename S, bool WALLS, int I>
__device__ __forceinline__ float pull_q(const S* __restrict__ src, const Box& b, const Nbr& q, int x, int y, int z,
                                        uint32_t self, float lx, float ly, float lz) {
    uint32_t cell;
    const bool wall = pull_source<I>(b, q, x, y, z, cell);
    if (!WALLS || !wall) return ldg_l2pf<S>(src + (size_t)I * b.n + cell);
    // half-way bounce-back; the lid term 6 w c.u_lid is 6 c.u_lid in units of w
    float v = Store<S>::load(src + (size_t)opp_of(I) * b.n + self);
    if (cy_of(I) < 0 && q.wyp) v += 6.f * ((float)cx_of(I) * lx + (float)cy_of(I) * ly + (float)cz_of(I) * lz);
    return v;
}

// At most 128 threads and 72 registers (7 CTAs, 28 warps per SM; 78 registers
// left 6): the kernel waits on its 38 pulls, and the extra warps hide more of
// that latency.
template <typename S, bool WALLS>
__global__ void __launch_bounds__(ZPAIR_MAX_THREADS, 7) fluid_step_zpair_kernel(const S* __restrict__ src,
                                                                              S* __restrict__ dst, FluidArgs p) {
    const Box& b = p.box;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= b.nx) return;
    const int y = blockIdx.y, za = 2 * (int)blockIdx.z;
    const bool two = za + 1 < b.nz;
    const int zb = two ? za + 1 : za;
    const uint32_t sa = ((uint32_t)za * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const uint32_t sb = ((uint32_t)zb * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr qa = make_nbr(b, x, y, za), qb = make_nbr(b, x, y, zb);
    const float lx = (float)p.lid[0], ly = (float)p.lid[1], lz = (float)p.lid[2];
    P2 f[Q];
#define LBM_ZP(I)                                                                                 \
    f[I] = P2(pull_q<S, WALLS, I>(src, b, qa, x, y, za, sa, lx, ly, lz),                          \
              pull_q<S, WALLS, I>(src, b, qb, x, y, zb, sb, lx, ly, lz));
    LBM_ZP(0) LBM_ZP(1) LBM_ZP(2) LBM_ZP(3) LBM_ZP(4) LBM_ZP(5) LBM_ZP(6) LBM_ZP(7) LBM_ZP(8) LBM_ZP(9)
    LBM_ZP(10) LBM_ZP(11) LBM_ZP(12) LBM_ZP(13) LBM_ZP(14) LBM_ZP(15) LBM_ZP(16) LBM_ZP(17) LBM_ZP(18)
#undef LBM_ZP
    const Moments<P2> m = moments19_q(f);
    const Macro<P2> a = fluid_macro(m, P2((float)p.g[0]), P2((float)p.g[1]), P2((float)p.g[2]));
    collide_fluid<P2, true>(f, m, a, P2((float)p.omega));
#define LBM_ZS(I)                                                        \
    {                                                                    \
        Store<S>::store(dst + (size_t)I * b.n + sa, f[I].v.x);           \
        if (two) Store<S>::store(dst + (size_t)I * b.n + sb, f[I].v.y);  \
    }
    LBM_ZS(0) LBM_ZS(1) LBM_ZS(2) LBM_ZS(3) LBM_ZS(4) LBM_ZS(5) LBM_ZS(6) LBM_ZS(7) LBM_ZS(8) LBM_ZS(9)
    LBM_ZS(10) LBM_ZS(11) LBM_ZS(12) LBM_ZS(13) LBM_ZS(14) LBM_ZS(15) LBM_ZS(16) LBM_ZS(17) LBM_ZS(18)
#undef LBM_ZS
}

// ---------------------------------------------------------------------------
// TMA-staged persistent step.  Work unit = one x-row (y, z).  For each row the
// 19 source rows (plane i at (y - c_iy, z - c_iz), whole rows of nx values) are
// fetched into shared memory by 1D bulk copies that complete on the stage's
// mbarrier; `stages` rows are in flight per CTA, so the bytes in flight do not
// cost registers.  x-shifts and the periodic x-wrap are index arithmetic in
// shared memory; pulls from behind a wall fall back to the node's own opposite
// population in global memory.  Waits are bounded: on a timeout the CTA writes
// LBM_ERR_TIMEOUT to `status`, drains its outstanding copies (bounded) and
// returns.  Requires nx * sizeof(S) to be a multiple of 16 bytes.
constexpr unsigned long long TMA_WAIT_NS = 1000000000ull;

// Issue the bulk copies of row r's 19 source rows into `stage` (warp 0: lane 0
// registers the expected bytes, then lanes 0..18 issue one copy each).
template <typename S, bool WALLS>
__device__ __forceinline__ void issue_row(const S* __restrict__ src, const Box& b, S* stage, uint64_t* bar, long r,
                                          int lane) {
    const int y = (int)(r % b.ny), z = (int)(r / b.ny);
    const Nbr q = make_nbr(b, 0, y, z);
    const uint32_t row_bytes = (uint32_t)b.nx * (uint32_t)sizeof(S);
    // lane i < 19 handles direction i; a source row behind a wall is not fetched
    int i = lane < Q ? lane : 0;
    const int cy = cy_of_rt(i), cz = cz_of_rt(i);
    const bool wall = WALLS && ((cy > 0 && q.wym) || (cy < 0 && q.wyp) || (cz > 0 && q.wzm) || (cz < 0 && q.wzp));
    const bool mine = lane < Q && !wall;
    const unsigned fetch = __ballot_sync(0xffffffffu, mine);
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)__popc(fetch) * row_bytes);
    __syncwarp();
    if (mine) {
        const int sy = cy == 0 ? y : (cy > 0 ? q.ym : q.yp);
        const int sz = cz == 0 ? z : (cz > 0 ? q.zm : q.zp);
        bulk_g2s(stage + (size_t)i * b.nx, src + (size_t)i * b.n + ((size_t)sz * b.ny + sy) * b.nx, row_bytes, bar);
    }
}

template <typename S, typename C, bool WALLS, int I>
__device__ __forceinline__ C pull_staged(const S* __restrict__ stage, const S* __restrict__ src, const Box& b,
                                         const Nbr& q, int x, int y, int z, uint32_t self, C lx, C ly, C lz) {
    constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
    if (WALLS) {
        const bool wall = (cx > 0 && q.wxm) || (cx < 0 && q.wxp) || (cy > 0 && q.wym) || (cy < 0 && q.wyp) ||
                          (cz > 0 && q.wzm) || (cz < 0 && q.wzp);
        if (wall) {
            C v = load_shifted<S, C, opp_of(I)>(src + (size_t)opp_of(I) * b.n + self);
            if (cy < 0 && q.wyp) v += (C)(6.0 * w_of(I)) * ((C)cx * lx + (C)cy * ly + (C)cz * lz);
            return v;
        }
    }
    const int sx = cx == 0 ? x : (cx > 0 ? q.xm : q.xp);
    C v = (C)Store<S>::to_float(stage[(size_t)I * b.nx + sx]);
    if (Store<S>::scaled) v *= (C)w_of(I);
    return v;
}

template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(256, 4) fluid_step_tma_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                                FluidArgs p, int stages, int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem[];
    const Box& b = p.box;
    const size_t stage_elems = (size_t)Q * b.nx;
    S* sbuf = reinterpret_cast<S*>(smem);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (((size_t)stages * stage_elems * sizeof(S) + 15) & ~size_t(15)));
    const long rows = (long)b.ny * b.nz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int k = 0; k < stages; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (warp == 0) {
        fence_proxy_async();
        for (int k = 0; k < stages; ++k) {
            const long r = blockIdx.x + (long)k * gridDim.x;
            if (r < rows) issue_row<S, WALLS>(src, b, sbuf + k * stage_elems, &bars[k], r, lane);
        }
    }
    const C lx = (C)p.lid[0], ly = (C)p.lid[1], lz = (C)p.lid[2];
    const C gx = (C)p.g[0], gy = (C)p.g[1], gz = (C)p.g[2], om = (C)p.omega;
    long k = 0;
    for (long r = blockIdx.x; r < rows; r += gridDim.x, ++k) {
        const int st = (int)(k % stages);
        const uint32_t parity = (uint32_t)((k / stages) & 1);
        // every thread waits (bounded) for the stage; the vote makes the
        // continue/stop decision uniform across the CTA
        const bool ready = mbar_wait_bounded(&bars[st], parity, TMA_WAIT_NS);
        if (!__syncthreads_and(ready)) {
            if (threadIdx.x == 0) {
                atomicExch(status, (int)LBM_ERR_TIMEOUT);
                // drain the copies this CTA still has in flight (bounded)
                for (long k2 = k; k2 < k + stages; ++k2) {
                    const long r2 = blockIdx.x + k2 * gridDim.x;
                    if (r2 < rows) mbar_wait_bounded(&bars[k2 % stages], (uint32_t)((k2 / stages) & 1), TMA_WAIT_NS);
                }
            }
            return;
        }
        const S* stage = sbuf + st * stage_elems;
        const int y = (int)(r % b.ny), z = (int)(r / b.ny);
        for (int x = threadIdx.x; x < b.nx; x += blockDim.x) {
            const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
            const Nbr q = make_nbr(b, x, y, z);
            C f[Q];
#define LBM_PS(I) f[I] = pull_staged<S, C, WALLS, I>(stage, src, b, q, x, y, z, self, lx, ly, lz);
            LBM_PS(0) LBM_PS(1) LBM_PS(2) LBM_PS(3) LBM_PS(4) LBM_PS(5) LBM_PS(6) LBM_PS(7) LBM_PS(8) LBM_PS(9)
            LBM_PS(10) LBM_PS(11) LBM_PS(12) LBM_PS(13) LBM_PS(14) LBM_PS(15) LBM_PS(16) LBM_PS(17) LBM_PS(18)
#undef LBM_PS
            const Moments<C> m = moments19(f);
            const Macro<C> a = fluid_macro(m, gx, gy, gz);
            collide_fluid<C>(f, m, a, om);
            scatter19<S, C>(dst, b.n, self, f);
        }
        __syncthreads();  // stage `st` fully read
        if (warp == 0) {
            const long r2 = r + (long)stages * gridDim.x;
            if (r2 < rows) {
                fence_proxy_async();
                issue_row<S, WALLS>(src, b, sbuf + st * stage_elems, &bars[st], r2, lane);
            }
        }
    }
}

// Equilibrium initialisation of a z-slab from FP64 fields (rho, ux, uy, uz
// planes of nx*ny*nzs values), or of the uniform rest state.
template <typename S, typename C>
__global__ void fluid_init_kernel(S* __restrict__ dst, const double* __restrict__ slab, Box b, int z0, int nzs,
                                  bool uniform) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, zs = blockIdx.z;
    if (x >= b.nx || zs >= nzs) return;
    const size_t m = (size_t)b.nx * b.ny * nzs;
    const size_t k = ((size_t)zs * b.ny + y) * b.nx + x;
    const uint32_t self = ((uint32_t)(z0 + zs) * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    C rho = (C)1, drho = (C)0, ux = (C)0, uy = (C)0, uz = (C)0;
    if (!uniform) {
        drho = (C)(slab[k] - 1.0);  // the shift is taken in FP64
        rho = (C)slab[k];
        ux = (C)slab[m + k];
        uy = (C)slab[2 * m + k];
        uz = (C)slab[3 * m + k];
    }
    C f[Q];
    equilibrium_shifted<C>(rho, drho, ux, uy, uz, f);
    conserve_mass<C>(f, drho);
    scatter19<S, C>(dst, b.n, self, f);
}

// Moments of the gathered state for a z-slab: rho, u (with +F/2).  REG: the
// regularized walls' rebuilt populations on the wall rows.
template <typename S, typename C, bool WALLS, bool REG = false>
__global__ void fluid_fields_kernel(const S* __restrict__ src, double* __restrict__ slab, FluidArgs p, int z0,
                                    int nzs) {
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
    if (REG)
        gather_regularized<S, C>(src, p, q, x, y, z, self, f);
    else
        gather19<S, C, WALLS>(src, b, q, x, y, z, self, (C)p.lid[0], (C)p.lid[1], (C)p.lid[2], f);
    const Moments<C> mo = moments19(f);
    const Macro<C> a = fluid_macro(mo, (C)p.g[0], (C)p.g[1], (C)p.g[2]);
    slab[k] = (double)a.rho;
    slab[m + k] = (double)a.ux;
    slab[2 * m + k] = (double)a.uy;
    slab[3 * m + k] = (double)a.uz;
}

template <typename S, typename C, bool WALLS, bool REG = false>
__global__ void __launch_bounds__(RED_THREADS) fluid_reduce_kernel(const S* __restrict__ src, FluidArgs p,
                                                                   C* __restrict__ uprev, bool have_prev,
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
            if (REG)
                gather_regularized<S, C>(src, p, q, x, y, z, self, f);
            else
                gather19<S, C, WALLS>(src, b, q, x, y, z, self, (C)p.lid[0], (C)p.lid[1], (C)p.lid[2], f);
            const Moments<C> mo = moments19(f);
            const Macro<C> a = fluid_macro(mo, (C)p.g[0], (C)p.g[1], (C)p.g[2]);
            reduce_node<C>(acc, a.rho, a.ux, a.uy, a.uz, uprev, b.n, self, have_prev, record);
        }
    }
    block_reduce_store(acc, partials);
}

// ---------------------------------------------------------------------------
static FluidArgs fluid_args(const lbm_ctx* c) {
    FluidArgs p;
    p.box = c->box;
    p.omega = c->relax.omega;
    for (int a = 0; a < 3; ++a) {
        p.g[a] = c->forcing.g[a];
        p.lid[a] = (c->box.periodic & 2u) ? 0.0 : c->grid.lid_u[a];
    }
    return p;
}

template <typename S>
static constexpr bool is16() {
    return sizeof(S) == 2;
}

// Shared-memory budget of one CTA of the staged kernel: the opt-in maximum per
// block (227 KB) with one CTA per SM, else an even share of the SM's 228 KB
// less the 1 KB the runtime reserves per CTA; 256 bytes are kept for the
// kernel's static shared memory.
constexpr size_t SMEM_PER_BLOCK_OPTIN = 227 * 1024;
constexpr size_t SMEM_PER_SM = 228 * 1024;

static size_t tma_stage_bytes(const lbm_ctx* c) { return (size_t)Q * c->box.nx * c->elem; }
static size_t tma_smem_bytes(const lbm_ctx* c, int stages) {
    return (((size_t)stages * tma_stage_bytes(c) + 15) & ~size_t(15)) + (size_t)stages * 8;
}

int fluid_tma_max_stages(const lbm_ctx* c, int ctas) {
    if (c->physics != LBM_PHYS_FLUID || c->q != 19 || c->grid.wall_model != LBM_WALL_BOUNCE_BACK ||
        c->relax.moment_space != LBM_MOMENTS_CENTRAL || ctas < 1 || ctas > 4)
        return 0;
    if (((size_t)c->box.nx * c->elem) % 16 != 0 || c->box.nx < 32) return 0;
    const size_t budget = (ctas == 1 ? SMEM_PER_BLOCK_OPTIN : SMEM_PER_SM / (size_t)ctas - 1024) - 256;
    int st = 0;
    while (st < 8 && tma_smem_bytes(c, st + 1) <= budget) ++st;
    return st >= 2 ? st : 0;
}

template <typename S, typename C, bool WALLS>
static cudaError_t launch_tma(lbm_ctx* c, const S* src, S* dst, const FluidArgs& p) {
    const int stages = c->tma_stages;
    const size_t smem = tma_smem_bytes(c, stages);
    static int max_dynamic = -1;  // per instantiation: opt-in minus the static shared memory
    if (max_dynamic < 0) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, fluid_step_tma_kernel<S, C, WALLS>);
        if (e != cudaSuccess) return e;
        const int dyn = (int)SMEM_PER_BLOCK_OPTIN - (int)fa.sharedSizeBytes;
        e = cudaFuncSetAttribute(fluid_step_tma_kernel<S, C, WALLS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dyn);
        if (e != cudaSuccess) return e;
        max_dynamic = dyn;
    }
    if ((long)smem > (long)max_dynamic) return cudaErrorInvalidValue;
    const long rows = (long)c->box.ny * c->box.nz;
    long grid = (long)c->sms * c->tma_ctas;
    if (grid > rows) grid = rows;
    int block = ((c->box.nx + 31) / 32) * 32;
    if (block > 256) block = 256;
    fluid_step_tma_kernel<S, C, WALLS><<<(unsigned)grid, block, smem, c->stream>>>(src, dst, p, stages, c->status);
    return cudaSuccess;
}

template <typename S, typename C>
static cudaError_t step_t(lbm_ctx* c, long n, bool dry) {
    const FluidArgs p = fluid_args(c);
    const bool walls = (c->box.periodic & 7u) != 7u;
    const int bx = c->block_x;
    if (c->relax.moment_space == LBM_MOMENTS_RAW) {
        const dim3 grid = step_grid(c->box, bx);
        for (long s = 0; s < n; ++s) {
            const S* src = (const S*)c->buf[c->cur];
            S* dst = (S*)c->buf[c->cur ^ 1];
            if (walls)
                fluid_step_kernel<S, C, true, true><<<grid, bx, 0, c->stream>>>(src, dst, p);
            else
                fluid_step_kernel<S, C, false, true><<<grid, bx, 0, c->stream>>>(src, dst, p);
            if (!dry) c->cur ^= 1;
        }
        return cudaGetLastError();
    }
    const bool reg = c->grid.wall_model == LBM_WALL_REGULARIZED;
    const bool channel = (c->box.periodic & 7u) == 5u && c->box.ny >= 3;
    if (channel && (reg || c->variant == 0)) {
        const unsigned gx = (unsigned)((c->box.nx + bx - 1) / bx);
        const dim3 inner(gx, (unsigned)(c->box.ny - 2), (unsigned)c->box.nz), rows(gx, 2u, (unsigned)c->box.nz);
        for (long s = 0; s < n; ++s) {
            const S* src = (const S*)c->buf[c->cur];
            S* dst = (S*)c->buf[c->cur ^ 1];
            fluid_step_interior_kernel<S, C><<<inner, bx, 0, c->stream>>>(src, dst, p);
            if (reg)
                fluid_step_wallrows_kernel<S, C, true><<<rows, bx, 0, c->stream>>>(src, dst, p);
            else
                fluid_step_wallrows_kernel<S, C, false><<<rows, bx, 0, c->stream>>>(src, dst, p);
            if (!dry) c->cur ^= 1;
        }
        return cudaGetLastError();
    }
    if (c->variant == 1 && c->tma_stages >= 2 && c->tma_stages <= fluid_tma_max_stages(c, c->tma_ctas)) {
        for (long s = 0; s < n; ++s) {
            const S* src = (const S*)c->buf[c->cur];
            S* dst = (S*)c->buf[c->cur ^ 1];
            cudaError_t e = walls ? launch_tma<S, C, true>(c, src, dst, p) : launch_tma<S, C, false>(c, src, dst, p);
            if (e != cudaSuccess) return e;
            if (!dry) c->cur ^= 1;
        }
        return cudaGetLastError();
    }
    const dim3 grid = step_grid(c->box, bx);
    const bool pair = is16<S>() && c->variant == 2 && (c->box.nx % 2 == 0);
    const bool zpair = is16<S>() && c->variant == 4;
    const dim3 grid2((unsigned)((c->box.nx / 2 + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)c->box.nz);
    const dim3 gridz(grid.x, grid.y, (unsigned)((c->box.nz + 1) / 2));
    for (long s = 0; s < n; ++s) {
        const S* src = (const S*)c->buf[c->cur];
        S* dst = (S*)c->buf[c->cur ^ 1];
        if constexpr (is16<S>()) {
            if (zpair) {
                if (walls)
                    fluid_step_zpair_kernel<S, true><<<gridz, bx, 0, c->stream>>>(src, dst, p);
                else
                    fluid_step_zpair_kernel<S, false><<<gridz, bx, 0, c->stream>>>(src, dst, p);
                if (!dry) c->cur ^= 1;
                continue;
            }
            if (pair) {
                if (walls)
                    fluid_step_pair_kernel<S, true><<<grid2, bx, 0, c->stream>>>(src, dst, p);
                else
                    fluid_step_pair_kernel<S, false><<<grid2, bx, 0, c->stream>>>(src, dst, p);
                if (!dry) c->cur ^= 1;
                continue;
            }
        }
        if (walls)
            fluid_step_kernel<S, C, true><<<grid, bx, 0, c->stream>>>(src, dst, p);
        else
            fluid_step_kernel<S, C, false><<<grid, bx, 0, c->stream>>>(src, dst, p);
        if (!dry) c->cur ^= 1;
    }
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t init_t(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform) {
    const int bx = c->block_x;
    dim3 grid((unsigned)((c->box.nx + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)nzs);
    fluid_init_kernel<S, C><<<grid, bx, 0, c->stream>>>((S*)c->buf[c->cur], slab, c->box, z0, nzs, uniform);
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t fields_t(lbm_ctx* c, double* slab, int z0, int nzs) {
    const FluidArgs p = fluid_args(c);
    const int bx = c->block_x;
    dim3 grid((unsigned)((c->box.nx + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)nzs);
    if (c->grid.wall_model == LBM_WALL_REGULARIZED)
        fluid_fields_kernel<S, C, true, true><<<grid, bx, 0, c->stream>>>((const S*)c->buf[c->cur], slab, p, z0, nzs);
    else if ((c->box.periodic & 7u) != 7u)
        fluid_fields_kernel<S, C, true><<<grid, bx, 0, c->stream>>>((const S*)c->buf[c->cur], slab, p, z0, nzs);
    else
        fluid_fields_kernel<S, C, false><<<grid, bx, 0, c->stream>>>((const S*)c->buf[c->cur], slab, p, z0, nzs);
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t reduce_t(lbm_ctx* c, bool record) {
    const FluidArgs p = fluid_args(c);
    if (c->grid.wall_model == LBM_WALL_REGULARIZED)
        fluid_reduce_kernel<S, C, true, true><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            (const S*)c->buf[c->cur], p, (C*)c->uprev, c->have_prev, record, c->partials);
    else if ((c->box.periodic & 7u) != 7u)
        fluid_reduce_kernel<S, C, true><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            (const S*)c->buf[c->cur], p, (C*)c->uprev, c->have_prev, record, c->partials);
    else
        fluid_reduce_kernel<S, C, false><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            (const S*)c->buf[c->cur], p, (C*)c->uprev, c->have_prev, record, c->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce_finalize(c);
}

cudaError_t fluid_step(lbm_ctx* c, long n, bool dry) {
    switch (c->prec) {
        case LBM_FP64: return step_t<double, double>(c, n, dry);
        case LBM_FP32: return step_t<float, float>(c, n, dry);
        case LBM_FP16_SHIFTED: return step_t<__half, float>(c, n, dry);
        case LBM_BF16_SHIFTED: return step_t<__nv_bfloat16, float>(c, n, dry);
    }
    return cudaErrorInvalidValue;
}
cudaError_t fluid_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform) {
    switch (c->prec) {
        case LBM_FP64: return init_t<double, double>(c, slab, z0, nzs, uniform);
        case LBM_FP32: return init_t<float, float>(c, slab, z0, nzs, uniform);
        case LBM_FP16_SHIFTED: return init_t<__half, float>(c, slab, z0, nzs, uniform);
        case LBM_BF16_SHIFTED: return init_t<__nv_bfloat16, float>(c, slab, z0, nzs, uniform);
    }
    return cudaErrorInvalidValue;
}
cudaError_t fluid_fields(lbm_ctx* c, double* slab, int z0, int nzs) {
    switch (c->prec) {
        case LBM_FP64: return fields_t<double, double>(c, slab, z0, nzs);
        case LBM_FP32: return fields_t<float, float>(c, slab, z0, nzs);
        case LBM_FP16_SHIFTED: return fields_t<__half, float>(c, slab, z0, nzs);
        case LBM_BF16_SHIFTED: return fields_t<__nv_bfloat16, float>(c, slab, z0, nzs);
    }
    return cudaErrorInvalidValue;
}
cudaError_t fluid_reduce(lbm_ctx* c, bool record) {
    switch (c->prec) {
        case LBM_FP64: return reduce_t<double, double>(c, record);
        case LBM_FP32: return reduce_t<float, float>(c, record);
        case LBM_FP16_SHIFTED: return reduce_t<__half, float>(c, record);
        case LBM_BF16_SHIFTED: return reduce_t<__nv_bfloat16, float>(c, record);
    }
    return cudaErrorInvalidValue;
}

// Deterministic final sum of the per-block partials (one block).
__global__ void reduce_finalize_kernel(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    __shared__ double sh[RED_THREADS][RED_WIDTH];
    double acc[RED_WIDTH];
#pragma unroll
    for (int k = 0; k < RED_WIDTH; ++k) acc[k] = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < RED_WIDTH; ++k) acc[k] += partials[(size_t)i * RED_WIDTH + k];
#pragma unroll
    for (int k = 0; k < RED_WIDTH; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < RED_WIDTH; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x < RED_WIDTH) out[threadIdx.x] = sh[0][threadIdx.x];
}

cudaError_t reduce_finalize(lbm_ctx* c) {
    reduce_finalize_kernel<<<1, RED_THREADS, 0, c->stream>>>(c->partials, RED_BLOCKS, c->result);
    return cudaGetLastError();
}

}  // namespace lbm
