// lbm_cnn.cu -- learned warm start: a small 3D convolutional network that maps
// (Reynolds number, node coordinates, lid mask) to the steady (rho, u) of the
// lid-driven cavity, trained on steady states produced by the solver; its
// prediction initialises the populations (f = f_eq of the predicted fields).
//
// Architecture (fixed): 4 layers of 3x3x3 convolutions with zero padding,
// 16 -> 32 -> 32 -> 32 -> 4 channels, ReLU after the first three (six layers
// predicted u slightly better, 0.050 against 0.054, but warm-started the
// solver less well: 55 % against 59 % mean wall-time reduction).  Activations
// and the weights used by the kernels are BF16, master weights, gradients and
// Adam moments FP32.  Activations are stored channel-chunked,
// [C/8][z][y][x][8] (8 channels = 16 bytes per node and chunk plane).
//
// Kernels:
//  - conv_tc: implicit GEMM on the tensor cores: tcgen05.mma (BF16 operands,
//    FP32 accumulators in TMEM).  A tile is a 128-node segment of an x-row;
//    per (dy, dz) the 130-node row (with its x-halo) of every channel chunk
//    is staged by 1D bulk copies of its contiguous runs, and the three
//    x-shifted taps read it through descriptor start offsets of 16 bytes
//    (unswizzled core matrices): 9 staged rows per tile instead of 27 boxes,
//    three rows per ring stage.  The same kernel runs the backward data pass
//    with the flipped, transposed weights.
//  - wgrad_tc: weight gradients on the tensor cores (rows x input channels as
//    M at one x-shift, output channels as N, voxels as K) from the same nine
//    staged rows per tile, with the bias gradients summed from the staged dY
//    tiles by the otherwise idle epilogue warps; one partial per CTA, summed
//    in a fixed order.
//  - adam: the optimiser step on the FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_internal.h"
#include "lbm_tc.cuh"

namespace cnn {

constexpr int NL = 4;
constexpr int C_IN_REAL = 16, C_OUT_REAL = 4;
// padded channel counts per layer boundary: input 16, hidden 32, output 16
constexpr int CH[NL + 1] = {16, 32, 32, 32, 16};
constexpr int CH_REAL[NL + 1] = {16, 32, 32, 32, 4};
constexpr float RHO_SCALE = 30.f;  // network output 0 = (rho - 1) * RHO_SCALE
constexpr float U_SCALE = 10.f;    // outputs 1..3 = u * U_SCALE (lid speed 0.1 -> 1)

constexpr int layer_params(int l) { return 27 * CH_REAL[l + 1] * CH_REAL[l] + CH_REAL[l + 1]; }
constexpr int total_params() {
    int n = 0;
    for (int l = 0; l < NL; ++l) n += layer_params(l);
    return n;
}

struct Shape {
    int nx, ny, nz;
    long P;
};

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ uint32_t bf_pack(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

// ---------------------------------------------------------------------------
// Tensor-core convolution (tcgen05, TMEM accumulators, bulk-copy staging).
//
// Implicit GEMM per tile of 128 voxels, a segment x0 .. x0 + 127 of the x-row
// (y, z): D[x][co] = sum over the 27 taps of A_tap[x][ci] W[tap][co][ci].
// For each (dy, dz) the row (y + dy, z + dz), nodes x0 - 1 .. x0 + 128 of
// every channel chunk, is staged as [chunk][130 cells][8 channels]: in the
// channel-chunked activation layout each chunk's run of the row is contiguous
// in memory, so one 1D bulk copy per chunk moves it whole (full 128-byte
// lines, where a tensor-map box with 16-byte rows moved 32-byte sectors half
// used).  Cells outside the grid are zeros written by the producer warp (the
// x-halo cells at the two ends; whole rows outside in y or z), which is the
// convolution's zero padding.  In that layout a K-major operand is a run of
// unswizzled core matrices (8 nodes x 16 bytes, contiguous), so the tap dx
// reads the same row from a start 16 (dx + 1) bytes on (leading offset = the
// chunk stride, stride offset = 128 bytes).  The weights are K-major in the
// TMA's 64-byte (CI = 32) or 32-byte (CI = 16) swizzle and stay in shared
// memory for the CTA's life.
//
// Roles (192 threads): warp 0 stages rows into a ring of NSTAGE stages of
// three rows each, one hand-off per stage (lane 0 waits and arms the stage,
// lanes 0 .. 3 CI/8 - 1 issue one row chunk's copy each, the warp writes the
// zero cells; when a row is one tile its halo cells never change, so the ring
// is zeroed once and only rows outside the grid are written over); warp 1
// allocates TMEM and its lane 0 issues the MMAs (M = 128, N = CO, K = 16) into
// one of two TMEM accumulators; warps 2-5 read the finished accumulator (each
// warp its 32-lane quarter: one voxel per thread, CO columns), apply the
// epilogue and store.  Every wait is bounded (TC_WAIT_NS); on expiry the
// kernel records LBM_ERR_TIMEOUT in *status, the other roles stop, the copies
// and MMAs in flight are drained (bounded) and TMEM is freed.
constexpr int TILE_M = 128;
constexpr int ROW_NODES = TILE_M + 2;       // a staged row: the tile and its x-halo
constexpr int ROW_CHUNK = ROW_NODES * 16;  // one channel chunk of a staged row (bytes)
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;

// Tiles are 128-node segments of x-rows: ntx segments per row, ny * nz rows.
struct TileGeom {
    int nx, ny, nz;
    int ntx;
    int ntiles;
    long P;  // nodes (chunk-plane stride)
};

__device__ __forceinline__ void tile_origin(const TileGeom& g, int t, int& x0, int& y0, int& z0) {
    x0 = (t % g.ntx) * TILE_M;
    y0 = (t / g.ntx) % g.ny;
    z0 = t / (g.ntx * g.ny);
}

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
    const uint32_t a = lbm::smem_u32(p);
    return p + (((a + 1023u) & ~1023u) - a);
}

// Wait for phase `parity` of `bar`, giving up when another role aborted or the
// deadline passed (then recording the timeout).
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status) {
    if (lbm::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = lbm::global_ns();
    while (!lbm::mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (lbm::global_ns() - t0 > TC_WAIT_NS) {
            *abort_flag = 1;
            atomicExch(status, (int)LBM_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}
// Bounded wait that ignores the abort flag (draining before exit).
__device__ __forceinline__ void tc_drain(uint64_t* bar, uint32_t parity) {
    lbm::mbar_wait_bounded(bar, parity, TC_WAIT_NS);
}
// Lane 0 waits, the warp learns the outcome.
__device__ __forceinline__ bool tc_wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status,
                                             int lane) {
    bool ok = false;
    if (lane == 0) ok = tc_wait(bar, parity, abort_flag, status);
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// The in-grid run of a staged row: cells c0 .. c0 + n - 1 of 0 .. 129 hold
// nodes x0 - 1 + cell of row (y, z), starting at node index `src`; n = 0 when
// the row lies outside the grid in y or z.
struct RowRun {
    int c0, n;
    long src;
};

__device__ __forceinline__ RowRun row_run(const TileGeom& g, int x0, int y, int z) {
    RowRun r{0, 0, 0};
    if (y < 0 || y >= g.ny || z < 0 || z >= g.nz) return r;
    const int xa = max(x0 - 1, 0), xb = min(x0 + TILE_M + 1, g.nx);
    r.c0 = xa - (x0 - 1);
    r.n = xb - xa;
    r.src = ((long)z * g.ny + y) * g.nx + xa;
    return r;
}

// Warp-wide: write the zero cells of a staged row of NCH chunks (all of it
// when it lies outside the grid; else the x-halo cell before the run when x0 =
// 0 and the cell after it when the run ends at the grid's edge).  Cells
// further right only feed nodes beyond the edge, whose outputs are discarded
// (convolution) or whose gradient is zero (weight gradient).  Generic stores,
// made visible to the tensor cores' async proxy by the fence the caller runs.
template <int NCH>
__device__ __forceinline__ void zero_row_cells(uint8_t* slot, const RowRun& r, int lane) {
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    if (r.n == 0) {
        for (int i = lane; i < NCH * ROW_NODES; i += 32) reinterpret_cast<uint4*>(slot)[i] = z;
        return;
    }
    if (lane < NCH) {
        if (r.c0 > 0) reinterpret_cast<uint4*>(slot + lane * ROW_CHUNK)[0] = z;
        if (r.c0 + r.n < ROW_NODES) reinterpret_cast<uint4*>(slot + lane * ROW_CHUNK)[r.c0 + r.n] = z;
    }
}

// The bulk copy of chunk c of a staged row's in-grid run.
__device__ __forceinline__ void copy_row_chunk(uint8_t* slot, const __nv_bfloat16* X, long P, const RowRun& r, int c,
                                               uint64_t* bar) {
    if (r.n > 0)
        lbm::bulk_g2s(slot + c * ROW_CHUNK + r.c0 * 16, X + ((size_t)c * P + r.src) * 8, (uint32_t)r.n * 16u, bar);
}

// A ring stage holds RPS staged rows (RPS = 3: the rows dy = -1, 0, 1 of one
// dz), handed from the producer to the MMAs by one barrier.
template <int CI, int CO, int NSTAGE, int RPS>
struct ConvLayout {
    static constexpr int A_BYTES = (CI / 8) * ROW_CHUNK;          // a staged row, all chunks
    static constexpr int A_STRIDE = (A_BYTES + 127) / 128 * 128;  // row slots on 128-byte boundaries
    static constexpr int STAGE_BYTES = RPS * A_STRIDE;
    static constexpr int W_BYTES = 27 * CO * CI * 2;
    static constexpr int A_OFF = (W_BYTES + 1023) / 1024 * 1024;
    static constexpr int BAR_OFF = (A_OFF + NSTAGE * STAGE_BYTES + 7) / 8 * 8;
    static constexpr int NBAR = 2 * NSTAGE + 6;  // full, empty, tmem full x2, tmem empty x2, weights, drain
    static constexpr int BYTES = BAR_OFF + NBAR * 8 + 16 + 1024;  // + TMEM slot, abort flag, alignment slack
    static constexpr uint32_t TCOLS = 2 * CO <= 32 ? 32 : 64;       // two accumulators of CO columns
    static constexpr uint32_t SWZ_W = CI == 32 ? tc::SW_64B : tc::SW_32B;
    static constexpr uint32_t IDESC = tc::idesc_bf16_f32(TILE_M, CO, false, false);
    static_assert(A_OFF % 1024 == 0 && A_STRIDE % 128 == 0, "weights on the swizzle period, slots 128-byte aligned");
    static_assert(9 % RPS == 0, "a tile's nine rows fill whole stages");
    static_assert(RPS * (CI / 8) <= 32, "one producer lane per row chunk of a stage");
};

constexpr int CONV_STAGES = 2;
constexpr int CONV_RPS = 3;

// EPI: 0 = +bias, ReLU, BF16 out (chunked); 1 = +bias, FP32 out [P][4] (the
// output layer's real channels); 2 = zero where `gate` (this layer's forward
// activation, chunked) is not positive, BF16 out (chunked), no bias.
template <int CI, int CO, int EPI>
__global__ void __launch_bounds__(192, 2) conv_tc(const __nv_bfloat16* __restrict__ X,
                                               const __grid_constant__ CUtensorMap mapW, const float* __restrict__ bias,
                                               void* __restrict__ Y, const __nv_bfloat16* __restrict__ gate,
                                               TileGeom g, int* status) {
    using Lay = ConvLayout<CI, CO, CONV_STAGES, CONV_RPS>;
    constexpr int RPS = CONV_RPS;
    constexpr int NSTAGE = CONV_STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint8_t* sW = sm;
    uint8_t* sA = sm + Lay::A_OFF;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + Lay::BAR_OFF);
    uint64_t* empty = full + NSTAGE;
    uint64_t* tfull = empty + NSTAGE;
    uint64_t* tempty = tfull + 2;
    uint64_t* wfull = tempty + 2;
    uint64_t* drain = wfull + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Rows of one tile: the copies always fill cells 1 .. nx, so the halo
    // cells stay as zeroed here; only rows outside the grid are written over.
    const bool fixed_halo = g.ntx == 1;
    if (fixed_halo) {
        for (int i = threadIdx.x; i < NSTAGE * Lay::STAGE_BYTES / 16; i += blockDim.x)
            reinterpret_cast<uint4*>(sA)[i] = make_uint4(0u, 0u, 0u, 0u);
        lbm::fence_proxy_async();
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            lbm::mbar_init(&full[s], 1);
            lbm::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            lbm::mbar_init(&tfull[a], 1);
            lbm::mbar_init(&tempty[a], 4);  // one arrival per epilogue warp
        }
        lbm::mbar_init(wfull, 1);
        lbm::mbar_init(drain, 1);
        *abort_flag = 0;
        lbm::fence_barrier_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tslot, Lay::TCOLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // ---- producer warp: 9 staged rows per tile, RPS per stage ----
        if (lane == 0) {
            tc::prefetch_map(&mapW);
            lbm::mbar_arrive_expect_tx(wfull, Lay::W_BYTES);
            tc::tma_load_3d(sW, &mapW, 0, 0, 0, wfull);
        }
        int armed[NSTAGE];
        for (int s = 0; s < NSTAGE; ++s) armed[s] = -1;
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < g.ntiles && ok; t += gridDim.x) {
            int x0, y0, z0;
            tile_origin(g, t, x0, y0, z0);
            for (int r0 = 0; r0 < 9; r0 += RPS) {
                if (!tc_wait_warp(&empty[stage], phase ^ 1u, abort_flag, status, lane)) {
                    ok = false;
                    break;
                }
                uint8_t* st = sA + stage * Lay::STAGE_BYTES;
                uint32_t bytes = 0;
                bool zeroed = false;
#pragma unroll
                for (int j = 0; j < RPS; ++j) {
                    const int r = r0 + j;
                    const RowRun run = row_run(g, x0, y0 + r % 3 - 1, z0 + r / 3 - 1);
                    if (!fixed_halo || run.n == 0) {
                        zero_row_cells<CI / 8>(st + j * Lay::A_STRIDE, run, lane);
                        zeroed = true;
                    }
                    bytes += (uint32_t)((CI / 8) * run.n * 16);
                }
                if (zeroed) lbm::fence_proxy_async();
                __syncwarp();
                // lane 0 arms the stage, the lanes issue one row chunk each
                if (lane == 0) {
                    lbm::mbar_arrive_expect_tx(&full[stage], bytes);
                    armed[stage] = (int)phase;
                }
                __syncwarp();
                if (lane < RPS * (CI / 8)) {
                    const int j = lane / (CI / 8), r = r0 + j;
                    copy_row_chunk(st + j * Lay::A_STRIDE, X, g.P, row_run(g, x0, y0 + r % 3 - 1, z0 + r / 3 - 1),
                                   lane % (CI / 8), &full[stage]);
                }
                if (++stage == NSTAGE) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
        if (lane == 0) {
            // the copies land by themselves: wait for the last one of every stage
            for (int s = 0; s < NSTAGE; ++s)
                if (armed[s] >= 0) tc_drain(&full[s], (uint32_t)armed[s]);
            tc_drain(wfull, 0);
        }
    } else if (threadIdx.x == 32) {
        // ---- MMA issuer: the three taps (dx = -1, 0, 1) of each staged row ----
        if (tc_wait(wfull, 0, abort_flag, status)) {
            tc::fence_after_sync();
            int stage = 0;
            uint32_t phase = 0;
            int it = 0;
            bool ok = true;
            // descriptors built once, advanced by byte offsets per operand
            const uint64_t adesc0 = tc::smem_desc(lbm::smem_u32(sA), ROW_CHUNK, 128, tc::SW_NONE);
            const uint64_t wdesc0 = tc::smem_desc(lbm::smem_u32(sW), 16, 8 * CI * 2, Lay::SWZ_W);
            for (int t = blockIdx.x; t < g.ntiles && ok; t += gridDim.x, ++it) {
                const int acc = it & 1;
                if (!tc_wait(&tempty[acc], (((uint32_t)it >> 1) & 1u) ^ 1u, abort_flag, status)) break;
                tc::fence_after_sync();
                const uint32_t d = tbase + (uint32_t)(acc * CO);
                for (int r0 = 0; r0 < 9; r0 += RPS) {
                    if (!tc_wait(&full[stage], phase, abort_flag, status)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint64_t astage = tc::desc_advance(adesc0, stage * Lay::STAGE_BYTES);
                    const uint64_t wstage = tc::desc_advance(wdesc0, r0 * 3 * CO * CI * 2);  // tap 3 r0 onwards
#pragma unroll
                    for (int j = 0; j < RPS; ++j) {
#pragma unroll
                        for (int dxi = 0; dxi < 3; ++dxi) {
                            // tap (r0 + j) * 3 + dxi = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
#pragma unroll
                            for (int k = 0; k < CI / 16; ++k) {
                                const uint64_t ad =
                                    tc::desc_advance(astage, j * Lay::A_STRIDE + dxi * 16 + k * 2 * ROW_CHUNK);
                                const uint64_t bd = tc::desc_advance(wstage, (j * 3 + dxi) * CO * CI * 2 + k * 32);
                                tc::mma_bf16(d, ad, bd, Lay::IDESC, r0 > 0 || j > 0 || dxi > 0 || k > 0);
                            }
                        }
                    }
                    tc::mma_commit(&empty[stage]);
                    if (++stage == NSTAGE) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (ok) tc::mma_commit(&tfull[acc]);
            }
        }
        tc::mma_commit(drain);
        tc_drain(drain, 0);
    } else if (warp >= 2) {
        // ---- epilogue: TMEM -> registers -> global ----
        const int q = warp & 3;  // TMEM lanes 32q .. 32q + 31
        const int row = q * 32 + lane;
        float bvals[CO];
#pragma unroll
        for (int co = 0; co < CO; ++co) bvals[co] = (EPI == 2) ? 0.f : __ldg(bias + co);
        int it = 0;
        for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x, ++it) {
            const int acc = it & 1;
            const uint32_t tl = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * CO);
            if (!tc_wait_warp(&tfull[acc], ((uint32_t)it >> 1) & 1u, abort_flag, status, lane)) break;
            tc::fence_after_sync();
            uint32_t r[CO];
            if constexpr (CO == 32) tc::tmem_ld32(tl, r); else tc::tmem_ld16(tl, r);
            tc::tmem_ld_wait();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[acc]);
            float v[CO];
#pragma unroll
            for (int co = 0; co < CO; ++co) v[co] = __uint_as_float(r[co]);
            int x0, y0, z0;
            tile_origin(g, t, x0, y0, z0);
            const int x = x0 + row;
            if (x >= g.nx) continue;
            const long p = ((long)z0 * g.ny + y0) * g.nx + x;
#pragma unroll
            for (int co = 0; co < CO; ++co) v[co] += bvals[co];
            if (EPI == 0) {
#pragma unroll
                for (int co = 0; co < CO; ++co) v[co] = fmaxf(v[co], 0.f);
            }
            if (EPI == 2) {
#pragma unroll
                for (int j = 0; j < CO / 8; ++j) {
                    const uint4 gw = __ldg(reinterpret_cast<const uint4*>(gate) + (size_t)j * g.P + p);
                    const uint32_t w4[4] = {gw.x, gw.y, gw.z, gw.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        if (!(bf_lo(w4[h]) > 0.f)) v[8 * j + 2 * h] = 0.f;
                        if (!(bf_hi(w4[h]) > 0.f)) v[8 * j + 2 * h + 1] = 0.f;
                    }
                }
            }
            if (EPI == 1) {
                reinterpret_cast<float4*>(Y)[p] = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int j = 0; j < CO / 8; ++j)
                    reinterpret_cast<uint4*>(Y)[(size_t)j * g.P + p] =
                        make_uint4(bf_pack(v[8 * j], v[8 * j + 1]), bf_pack(v[8 * j + 2], v[8 * j + 3]),
                                   bf_pack(v[8 * j + 4], v[8 * j + 5]), bf_pack(v[8 * j + 6], v[8 * j + 7]));
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, Lay::TCOLS);
    }
}

// Weight gradient on the tensor cores: dW[tap][co][ci] = sum_p dY[p][co]
// X[p + off(tap)][ci].  Per tile (an x-row segment of 128 voxels) the nine
// rows (y + dy, z + dz) of X are staged as for the convolution, back to back
// ([row][chunk][130 cells][8 channels]), and the tile's dY as [chunk][128][8].
// D[(row, ci)][co] = A[(row, ci)][p] B[p][co] with M = 128 = TG rows x CI
// channels (TG = 4 for CI = 32, 8 for CI = 16) at one dx, the 128 voxels as
// K: both operands are MN-major runs of unswizzled core matrices (8 voxels x 8
// channels, 128 contiguous bytes), 8-voxel groups 128 bytes apart (leading
// offset) and channel chunks one chunk stride apart (stride offset); the
// chunks of consecutive staged rows continue at that stride, so one
// descriptor spans TG rows, and the tap dx starts 16 (dx + 1) bytes on.  The
// row groups start at rows 0, TG, ... with the last one moved back to end at
// row 8 (its rows already covered are discarded).  Every (row group, dx)
// accumulates in its own TMEM columns over all tiles of the CTA's contiguous
// range; the epilogue writes one partial per CTA, laid out [27][CO][CI],
// summed later in a fixed order.  The epilogue warps, idle until the end,
// also sum each staged dY tile over its voxels (the bias gradient, one
// partial per CTA beside the weights'), so a stage is free once the MMAs and
// those four warps are done with it.  On a tile cut by the grid's x-edge only
// the 16-voxel K-steps holding grid voxels are issued and dY is zeroed up to
// the step's end; the ring is zeroed at start so that every staged value the
// MMAs read is finite.
template <int CI, int CO>
struct WgLayout {
    static constexpr int TG = TILE_M / CI;
    static constexpr int NRG = (9 + TG - 1) / TG;  // row groups
    static constexpr int NGRP = 3 * NRG;           // (row group, dx) accumulators
    static constexpr int ROW = (CI / 8) * ROW_CHUNK;
    static constexpr int XB = 9 * ROW;
    static constexpr int YCHUNK = TILE_M * 16;
    static constexpr int YB = (CO / 8) * YCHUNK;
    static constexpr int STAGE = (XB + YB + 127) / 128 * 128;
    static constexpr int NSTAGE = CI == 32 ? 2 : 4;
    static constexpr int BAR_OFF = NSTAGE * STAGE;
    static constexpr int NBAR = 2 * NSTAGE + 2;  // full, empty, acc full, drain
    static constexpr int BYTES = BAR_OFF + NBAR * 8 + 16 + 4 * CO * 4 + 1024;  // + TMEM slot, flag, bias sums
    static constexpr int TCOLS_USED = NGRP * CO;
    static constexpr uint32_t TCOLS =
        TCOLS_USED <= 64 ? 64 : (TCOLS_USED <= 128 ? 128 : (TCOLS_USED <= 256 ? 256 : 512));
    static constexpr uint32_t IDESC = tc::idesc_bf16_f32(TILE_M, CO, true, true);
    static_assert(TG * CI == TILE_M && TCOLS_USED <= 512, "row groups must fill M = 128 within 512 TMEM columns");
    static_assert(XB % 16 == 0 && BYTES <= 227 * 1024, "staging must fit shared memory");
    __host__ __device__ static constexpr int group_row0(int rg) { return rg * TG < 9 - TG ? rg * TG : 9 - TG; }
};

template <int CI, int CO>
__global__ void __launch_bounds__(192) wgrad_tc(const __nv_bfloat16* __restrict__ X,
                                                const __nv_bfloat16* __restrict__ dY, float* __restrict__ partial,
                                                TileGeom g, int* status) {
    using Lay = WgLayout<CI, CO>;
    constexpr int NSTAGE = Lay::NSTAGE;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + Lay::BAR_OFF);
    uint64_t* empty = full + NSTAGE;
    uint64_t* accfull = empty + NSTAGE;
    uint64_t* drain = accfull + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    float* sbias = reinterpret_cast<float*>(tslot + 4);  // [4 warps][CO]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per = (g.ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t_begin = min(g.ntiles, (int)blockIdx.x * per), t_end = min(g.ntiles, t_begin + per);

    for (int i = threadIdx.x; i < NSTAGE * Lay::STAGE / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
    lbm::fence_proxy_async();
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            lbm::mbar_init(&full[s], 1);
            lbm::mbar_init(&empty[s], 5);  // the MMAs' commit and the four epilogue warps
        }
        lbm::mbar_init(accfull, 1);
        lbm::mbar_init(drain, 1);
        *abort_flag = 0;
        lbm::fence_barrier_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tslot, Lay::TCOLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // ---- producer warp: the nine X rows and dY of each tile ----
        int armed[NSTAGE];
        for (int s = 0; s < NSTAGE; ++s) armed[s] = -1;
        int stage = 0;
        uint32_t phase = 0;
        for (int t = t_begin; t < t_end; ++t) {
            if (!tc_wait_warp(&empty[stage], phase ^ 1u, abort_flag, status, lane)) break;
            int x0, y0, z0;
            tile_origin(g, t, x0, y0, z0);
            uint8_t* sx = sm + stage * Lay::STAGE;
            uint8_t* sy = sx + Lay::XB;
            uint32_t bytes = 0;
            for (int r = 0; r < 9; ++r) {
                const RowRun run = row_run(g, x0, y0 + r % 3 - 1, z0 + r / 3 - 1);
                zero_row_cells<CI / 8>(sx + r * Lay::ROW, run, lane);
                bytes += (uint32_t)((CI / 8) * run.n * 16);
            }
            const int nv = min(TILE_M, g.nx - x0);
            const int kend = (nv + 15) / 16 * 16;
            for (int i = lane; i < (CO / 8) * (kend - nv); i += 32)
                reinterpret_cast<uint4*>(sy + (i / (kend - nv)) * Lay::YCHUNK)[nv + i % (kend - nv)] =
                    make_uint4(0u, 0u, 0u, 0u);
            lbm::fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                lbm::mbar_arrive_expect_tx(&full[stage], bytes + (uint32_t)((CO / 8) * nv * 16));
                armed[stage] = (int)phase;
            }
            __syncwarp();
            // the 9 x CI/8 row-chunk copies and the CO/8 dY copies, spread over the lanes
            for (int i = lane; i < 9 * (CI / 8) + CO / 8; i += 32) {
                if (i < 9 * (CI / 8)) {
                    const int r = i / (CI / 8), c = i % (CI / 8);
                    copy_row_chunk(sx + r * Lay::ROW, X, g.P, row_run(g, x0, y0 + r % 3 - 1, z0 + r / 3 - 1), c,
                                   &full[stage]);
                } else {
                    const int c = i - 9 * (CI / 8);
                    const long p0 = ((long)z0 * g.ny + y0) * g.nx + x0;
                    lbm::bulk_g2s(sy + c * Lay::YCHUNK, dY + ((size_t)c * g.P + p0) * 8, (uint32_t)nv * 16u,
                                  &full[stage]);
                }
            }
            if (++stage == NSTAGE) {
                stage = 0;
                phase ^= 1u;
            }
        }
        if (lane == 0)
            for (int s = 0; s < NSTAGE; ++s)
                if (armed[s] >= 0) tc_drain(&full[s], (uint32_t)armed[s]);
    } else if (threadIdx.x == 32) {
        // ---- MMA issuer ----
        const uint64_t xdesc0 = tc::smem_desc(lbm::smem_u32(sm), 128, ROW_CHUNK, tc::SW_NONE);
        const uint64_t ydesc0 = tc::smem_desc(lbm::smem_u32(sm) + Lay::XB, 128, Lay::YCHUNK, tc::SW_NONE);
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int t = t_begin, it = 0; t < t_end; ++t, ++it) {
            if (!tc_wait(&full[stage], phase, abort_flag, status)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const int nk = (min(TILE_M, g.nx - (t % g.ntx) * TILE_M) + 15) / 16;
            const uint64_t xst = tc::desc_advance(xdesc0, stage * Lay::STAGE);
            const uint64_t yst = tc::desc_advance(ydesc0, stage * Lay::STAGE);
            // 16 voxels per K-step: 16 x 16 bytes into every chunk
            if (nk == TILE_M / 16) {
#pragma unroll
                for (int rg = 0; rg < Lay::NRG; ++rg)
#pragma unroll
                    for (int dxi = 0; dxi < 3; ++dxi)
#pragma unroll
                        for (int k = 0; k < TILE_M / 16; ++k)
                            tc::mma_bf16(tbase + (uint32_t)((rg * 3 + dxi) * CO),
                                         tc::desc_advance(xst, Lay::group_row0(rg) * Lay::ROW + dxi * 16 + k * 256),
                                         tc::desc_advance(yst, k * 256), Lay::IDESC, it > 0 || k > 0);
            } else {
                for (int rg = 0; rg < Lay::NRG; ++rg)
                    for (int dxi = 0; dxi < 3; ++dxi)
                        for (int k = 0; k < nk; ++k)
                            tc::mma_bf16(tbase + (uint32_t)((rg * 3 + dxi) * CO),
                                         tc::desc_advance(xst, Lay::group_row0(rg) * Lay::ROW + dxi * 16 + k * 256),
                                         tc::desc_advance(yst, k * 256), Lay::IDESC, it > 0 || k > 0);
            }
            tc::mma_commit(&empty[stage]);
            if (++stage == NSTAGE) {
                stage = 0;
                phase ^= 1u;
            }
        }
        if (ok) tc::mma_commit(accfull);
        tc::mma_commit(drain);
        tc_drain(drain, 0);
    } else if (warp >= 2) {
        // ---- epilogue: bias sums over the staged dY tiles, then the
        // accumulated groups -> this CTA's partial ----
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const int rsub = m / CI, ci = m % CI;
        float* out = partial + (size_t)blockIdx.x * (27 * CO * CI + CO);
        const bool have = t_end > t_begin;
        bool ok = true;
        float db[CO];
#pragma unroll
        for (int co = 0; co < CO; ++co) db[co] = 0.f;
        {
            int stage = 0;
            uint32_t phase = 0;
            for (int t = t_begin; t < t_end; ++t) {
                if (!tc_wait_warp(&full[stage], phase, abort_flag, status, lane)) {
                    ok = false;
                    break;
                }
                if (m < min(TILE_M, g.nx - (t % g.ntx) * TILE_M)) {
                    const uint4* yt = reinterpret_cast<const uint4*>(sm + stage * Lay::STAGE + Lay::XB);
#pragma unroll
                    for (int c = 0; c < CO / 8; ++c) {
                        const uint4 w = yt[c * (Lay::YCHUNK / 16) + m];
                        const uint32_t w4[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            db[8 * c + 2 * h] += bf_lo(w4[h]);
                            db[8 * c + 2 * h + 1] += bf_hi(w4[h]);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&empty[stage]);
                if (++stage == NSTAGE) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
#pragma unroll
        for (int co = 0; co < CO; ++co) {
            float v = db[co];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            db[co] = v;
        }
        if (lane == 0)
#pragma unroll
            for (int co = 0; co < CO; ++co) sbias[q * CO + co] = db[co];
        asm volatile("bar.sync 1, 128;" ::: "memory");  // the four epilogue warps
        if (q == 0 && lane < CO)
            out[27 * CO * CI + lane] = ok ? ((sbias[lane] + sbias[CO + lane]) + sbias[2 * CO + lane]) + sbias[3 * CO + lane]
                                          : 0.f;
        if (have && ok) {
            ok = tc_wait_warp(accfull, 0, abort_flag, status, lane);
            if (ok) tc::fence_after_sync();
        }
        if (ok) {
            for (int gi = 0; gi < Lay::NGRP; ++gi) {
                uint32_t r[CO];
                if (have) {
                    if constexpr (CO == 32)
                        tc::tmem_ld32(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(gi * CO), r);
                    else
                        tc::tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(gi * CO), r);
                    tc::tmem_ld_wait();
                } else {
#pragma unroll
                    for (int co = 0; co < CO; ++co) r[co] = 0u;
                }
                const int rg = gi / 3, dxi = gi % 3;
                const int row = Lay::group_row0(rg) + rsub;
                const bool owned = rg == 0 || row >= Lay::group_row0(rg - 1) + Lay::TG;
                if (owned) {
                    const int tap = row * 3 + dxi;
#pragma unroll
                    for (int co = 0; co < CO; ++co) out[((size_t)tap * CO + co) * CI + ci] = __uint_as_float(r[co]);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, Lay::TCOLS);
    }
}

__global__ void sum_partials(const float* __restrict__ partial, int nblocks, int width, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= width) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * width + i];
    out[i] = s;
}

// Master weights of layer l: [CO_real][CI_real][27] then bias [CO_real].
// Pack to the kernel layouts: fwd [27][CO][CI] and bwd-data [27][CI][CO]
// with the tap flipped (26 - tap); padding channels are zero.
__global__ void pack_weights(const float* __restrict__ master, __nv_bfloat16* __restrict__ wf,
                             __nv_bfloat16* __restrict__ wb, float* __restrict__ bias, int ci_r, int co_r, int ci_p,
                             int co_p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = 27 * co_p * ci_p;
    if (i < n) {
        const int tap = i / (co_p * ci_p), co = (i / ci_p) % co_p, ci = i % ci_p;
        const float v = (co < co_r && ci < ci_r) ? master[((size_t)co * ci_r + ci) * 27 + tap] : 0.f;
        wf[i] = __float2bfloat16_rn(v);
        wb[((size_t)(26 - tap) * ci_p + ci) * co_p + co] = __float2bfloat16_rn(v);
    }
    if (i < co_p) bias[i] = i < co_r ? master[(size_t)27 * co_r * ci_r + i] : 0.f;
}

// Gather the padded per-layer gradient into the master layout.
__global__ void unpack_grad(const float* __restrict__ g, float* __restrict__ master_grad, int ci_r, int co_r, int ci_p,
                            int co_p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = co_r * ci_r * 27;
    if (i < n) {
        const int co = i / (ci_r * 27), ci = (i / 27) % ci_r, tap = i % 27;
        master_grad[i] = g[((size_t)tap * co_p + co) * ci_p + ci];
    }
    if (i < co_r) master_grad[n + i] = g[(size_t)27 * co_p * ci_p + i];
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Input channels (16): r = (Re - 550)/450; the node-centre coordinates
// x, y, z scaled to [-1, 1]; lid = 1 on the top (+y) layer of nodes;
// cos(pi x/2), cos(pi y/2), cos(pi z/2) (vanishing at the walls);
// sin(pi x), sin(pi y), sin(pi z); cos(pi x), cos(pi y), cos(pi z); r^2;
// r (y + 1)/2.  The smooth coordinate functions let four 3x3x3 layers (a
// receptive field of 9 nodes) shape fields across the whole cavity.
__global__ void features(__nv_bfloat16* __restrict__ X0, Shape s, float re_n) {
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.P) return;
    const int x = (int)(p % s.nx), y = (int)((p / s.nx) % s.ny), z = (int)(p / ((long)s.nx * s.ny));
    float f[16];
    const float xn = 2.f * (x + 0.5f) / s.nx - 1.f;
    const float yn = 2.f * (y + 0.5f) / s.ny - 1.f;
    const float zn = 2.f * (z + 0.5f) / s.nz - 1.f;
    f[0] = re_n;
    f[1] = xn;
    f[2] = yn;
    f[3] = zn;
    f[4] = y == s.ny - 1 ? 1.f : 0.f;
    f[5] = cospif(0.5f * xn);
    f[6] = cospif(0.5f * yn);
    f[7] = cospif(0.5f * zn);
    f[8] = sinpif(xn);
    f[9] = sinpif(yn);
    f[10] = sinpif(zn);
    f[11] = cospif(xn);
    f[12] = cospif(yn);
    f[13] = cospif(zn);
    f[14] = re_n * re_n;
    f[15] = re_n * 0.5f * (yn + 1.f);
    // channel-chunked: channels 0..7 in chunk plane 0, 8..15 in plane 1
    uint4* o = reinterpret_cast<uint4*>(X0);
    o[p] = make_uint4(bf_pack(f[0], f[1]), bf_pack(f[2], f[3]), bf_pack(f[4], f[5]), bf_pack(f[6], f[7]));
    o[s.P + p] = make_uint4(bf_pack(f[8], f[9]), bf_pack(f[10], f[11]), bf_pack(f[12], f[13]), bf_pack(f[14], f[15]));
}

// Loss and its gradient: L = mean over voxels and the 4 real channels of
// (Y - T)^2 with T = [(rho - 1) RHO_SCALE, u U_SCALE] from FP64 fields
// (rho - 1 taken in FP64).  Grid-stride; each thread sums its squared errors
// in FP32, the block's in FP64 (one partial per block).
__global__ void __launch_bounds__(256) loss_grad(const float* __restrict__ Y, const double* __restrict__ rho,
                                                 const double* __restrict__ u, __nv_bfloat16* __restrict__ dY,
                                                 double* __restrict__ partial, Shape s) {
    __shared__ double sh[8];
    const float scale = 2.f / (4.f * (float)s.P);
    float l = 0.f;
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < s.P; p += (long)gridDim.x * blockDim.x) {
        const float4 y = reinterpret_cast<const float4*>(Y)[p];
        const float e0 = y.x - (float)((__ldg(rho + p) - 1.0) * RHO_SCALE);
        const float e1 = y.y - (float)(__ldg(u + p) * U_SCALE);
        const float e2 = y.z - (float)(__ldg(u + s.P + p) * U_SCALE);
        const float e3 = y.w - (float)(__ldg(u + 2 * s.P + p) * U_SCALE);
        l += (e0 * e0 + e1 * e1) + (e2 * e2 + e3 * e3);
        // channel-chunked gradient, chunk plane 0 (outputs 0..7); plane 1
        // (outputs 8..15) stays zero from the network's creation
        reinterpret_cast<uint4*>(dY)[p] =
            make_uint4(bf_pack(scale * e0, scale * e1), bf_pack(scale * e2, scale * e3), 0u, 0u);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void sum_double(const double* __restrict__ partial, long n, double* __restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// Prediction -> FP64 fields rho = 1 + y0/RHO_SCALE, u = y1..3/U_SCALE (planar).
__global__ void to_fields(const float* __restrict__ Y, double* __restrict__ rho, double* __restrict__ u, Shape s) {
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.P) return;
    rho[p] = 1.0 + (double)Y[p * 4 + 0] / RHO_SCALE;
    u[p] = (double)Y[p * 4 + 1] / U_SCALE;
    u[s.P + p] = (double)Y[p * 4 + 2] / U_SCALE;
    u[2 * s.P + p] = (double)Y[p * 4 + 3] / U_SCALE;
}

}  // namespace cnn

struct lbm_cnn {
    cnn::Shape s;
    cudaStream_t stream;
    lbm_alloc_fn alloc;
    lbm_free_fn release;
    void* user;
    float* master;    // FP32 master weights, all layers back to back
    float* grad;      // FP32 gradient, same layout
    float* adam_m;
    float* adam_v;
    long adam_t = 0;
    __nv_bfloat16* wf[cnn::NL];  // packed BF16 forward weights
    __nv_bfloat16* wb[cnn::NL];  // packed BF16 backward-data weights
    float* bias[cnn::NL];
    float* gpad[cnn::NL];        // padded per-layer gradient (summed partials)
    float* partial;              // weight-gradient partials
    __nv_bfloat16* act[cnn::NL]; // act[0] = input features, act[1..NL-1] hidden activations
    float* out;                  // [P][4] FP32 prediction
    __nv_bfloat16* dA[2];        // backward activations (ping-pong)
    __nv_bfloat16* dY4;          // output-layer gradient, 16 channels chunked (plane 1 always zero)
    double* rho_d;               // FP64 fields (prediction or target staging)
    double* u_d;
    double* lpart;               // loss partials
    double* lsum;
    int* status;                 // device status word (bounded-wait timeouts)
    int nsm = 0;                 // multiprocessors of the device
    int wg_blocks = 0;           // CTAs of the weight-gradient kernels (one partial each)
    cnn::TileGeom geom;          // 128-voxel tiles of the grid
    CUtensorMap m_wf[cnn::NL];   // forward weights [27][CO][CI]
    CUtensorMap m_wb[cnn::NL];   // backward-data weights [27][CI][CO] (layers 1..NL-1)
    std::string err;
};

namespace {

void* cnn_alloc(lbm_cnn* c, size_t bytes) {
    if (c->alloc) return c->alloc(bytes, (void*)c->stream, c->user);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void cnn_free(lbm_cnn* c, void* p) {
    if (!p) return;
    if (c->release)
        c->release(p, (void*)c->stream, c->user);
    else
        cudaFree(p);
}

size_t layer_offset(int l) {
    size_t o = 0;
    for (int k = 0; k < l; ++k) o += (size_t)cnn::layer_params(k);
    return o;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against libcuda).
EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// Tiles: 128-node segments of the x-rows.
cnn::TileGeom make_geom(int nx, int ny, int nz) {
    cnn::TileGeom g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.ntx = (nx + cnn::TILE_M - 1) / cnn::TILE_M;
    g.ntiles = g.ntx * ny * nz;
    g.P = (long)nx * ny * nz;
    return g;
}

// Packed weights [27][CO][CI] (BF16) as one 3D box holding all taps.
bool map_weights(CUtensorMap* m, const void* base, int CI, int CO) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)CI, (cuuint64_t)CO, 27};
    const cuuint64_t strides[2] = {(cuuint64_t)CI * 2, (cuuint64_t)CO * CI * 2};
    const cuuint32_t box[3] = {(cuuint32_t)CI, (cuuint32_t)CO, 27};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CI == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_maps(lbm_cnn* c) {
    bool ok = true;
    for (int l = 0; l < cnn::NL; ++l) {
        ok = ok && map_weights(&c->m_wf[l], c->wf[l], cnn::CH[l], cnn::CH[l + 1]);
        if (l > 0) ok = ok && map_weights(&c->m_wb[l], c->wb[l], cnn::CH[l + 1], cnn::CH[l]);
    }
    return ok;
}

template <int CI, int CO, int EPI>
cudaError_t conv(lbm_cnn* c, const __nv_bfloat16* X, const CUtensorMap& mapW, const float* bias, void* Y,
                 const __nv_bfloat16* gate) {
    const int smem = cnn::ConvLayout<CI, CO, cnn::CONV_STAGES, cnn::CONV_RPS>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(cnn::conv_tc<CI, CO, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int blocks = std::min(c->geom.ntiles, 2 * c->nsm);
    cnn::conv_tc<CI, CO, EPI><<<blocks, 192, smem, c->stream>>>(X, mapW, bias, Y, gate, c->geom, c->status);
    return cudaGetLastError();
}

template <int CI, int CO>
cudaError_t wgrad(lbm_cnn* c, const __nv_bfloat16* X, const __nv_bfloat16* dY, float* gpad) {
    const int smem = cnn::WgLayout<CI, CO>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(cnn::wgrad_tc<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cnn::wgrad_tc<CI, CO><<<c->wg_blocks, 192, smem, c->stream>>>(X, dY, c->partial, c->geom, c->status);
    const int width = 27 * CO * CI + CO;
    cnn::sum_partials<<<(width + 255) / 256, 256, 0, c->stream>>>(c->partial, c->wg_blocks, width, gpad);
    return cudaGetLastError();
}

// Device status word -> lbm_status (after a stream synchronisation).
lbm_status check_status(lbm_cnn* c, const char* where) {
    int st = 0;
    if (cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string(where) + ": status read failed";
        return LBM_ERR_CUDA;
    }
    if (st != 0) {
        c->err = std::string(where) + ": a tensor-core pipeline wait ran out of time";
        return (lbm_status)st;
    }
    return LBM_OK;
}

cudaError_t pack_all(lbm_cnn* c) {
    for (int l = 0; l < cnn::NL; ++l) {
        const int ci_p = cnn::CH[l], co_p = cnn::CH[l + 1];
        const int n = 27 * ci_p * co_p;
        cnn::pack_weights<<<(n + 255) / 256, 256, 0, c->stream>>>(c->master + layer_offset(l), c->wf[l], c->wb[l],
                                                                   c->bias[l], cnn::CH_REAL[l], cnn::CH_REAL[l + 1],
                                                                   ci_p, co_p);
    }
    return cudaGetLastError();
}

cudaError_t forward(lbm_cnn* c) {
    constexpr int L = cnn::NL;
    cudaError_t e = conv<16, 32, 0>(c, c->act[0], c->m_wf[0], c->bias[0], c->act[1], nullptr);
    for (int l = 1; l < L - 1 && e == cudaSuccess; ++l)
        e = conv<32, 32, 0>(c, c->act[l], c->m_wf[l], c->bias[l], c->act[l + 1], nullptr);
    if (e == cudaSuccess) e = conv<32, 16, 1>(c, c->act[L - 1], c->m_wf[L - 1], c->bias[L - 1], c->out, nullptr);
    return e;
}

// Backward from the output-layer gradient dY4 (16 channels, chunked); fills
// c->grad (weights and biases).
// The gradient of each hidden activation ping-pongs between dA[0] and dA[1].
cudaError_t backward(lbm_cnn* c, const __nv_bfloat16* dY4) {
    constexpr int L = cnn::NL;
    cudaError_t e = wgrad<32, 16>(c, c->act[L - 1], dY4, c->gpad[L - 1]);
    // gradient of act[L-1]: conv^T(dY, W_L) masked by act[L-1] > 0
    if (e == cudaSuccess) e = conv<16, 32, 2>(c, dY4, c->m_wb[L - 1], nullptr, c->dA[0], c->act[L - 1]);
    int cur = 0;
    for (int l = L - 2; l >= 1 && e == cudaSuccess; --l) {
        e = wgrad<32, 32>(c, c->act[l], c->dA[cur], c->gpad[l]);
        if (e == cudaSuccess) e = conv<32, 32, 2>(c, c->dA[cur], c->m_wb[l], nullptr, c->dA[cur ^ 1], c->act[l]);
        cur ^= 1;
    }
    if (e == cudaSuccess) e = wgrad<16, 32>(c, c->act[0], c->dA[cur], c->gpad[0]);
    for (int l = 0; l < cnn::NL && e == cudaSuccess; ++l) {
        const int n = 27 * cnn::CH_REAL[l] * cnn::CH_REAL[l + 1];
        cnn::unpack_grad<<<(n + 255) / 256, 256, 0, c->stream>>>(c->gpad[l], c->grad + layer_offset(l),
                                                                  cnn::CH_REAL[l], cnn::CH_REAL[l + 1], cnn::CH[l],
                                                                  cnn::CH[l + 1]);
        e = cudaGetLastError();
    }
    return e;
}

// Loss against FP64 target fields (device, planar rho [P], u [3P]); writes
// dY4 into its buffer and the loss sum into c->lsum.
cudaError_t loss(lbm_cnn* c, const double* rho, const double* u, __nv_bfloat16* dY4) {
    const long blocks = std::min<long>((c->s.P + 255) / 256, 4L * c->nsm);
    cnn::loss_grad<<<(unsigned)blocks, 256, 0, c->stream>>>(c->out, rho, u, dY4, c->lpart, c->s);
    cnn::sum_double<<<1, 256, 0, c->stream>>>(c->lpart, blocks, c->lsum);
    return cudaGetLastError();
}

lbm_status cnn_cuda_fail(lbm_cnn* c, cudaError_t e, const char* where) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    c->err = buf;
    return LBM_ERR_CUDA;
}

bool device_accessible(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = -1;
    cudaGetDevice(&dev);
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

// FP64 target fields for the loss: device pointers of this device are read in
// place; host pointers are staged into the network's buffers.
cudaError_t stage_fields(lbm_cnn* c, const double*& rho, const double*& u) {
    const size_t P = (size_t)c->s.P;
    cudaError_t e = cudaSuccess;
    if (!device_accessible(rho)) {
        e = cudaMemcpyAsync(c->rho_d, rho, P * 8, cudaMemcpyDefault, c->stream);
        rho = c->rho_d;
    }
    if (e == cudaSuccess && !device_accessible(u)) {
        e = cudaMemcpyAsync(c->u_d, u, 3 * P * 8, cudaMemcpyDefault, c->stream);
        u = c->u_d;
    }
    return e;
}

}  // namespace

extern "C" {

size_t lbm_cnn_param_count(void) { return (size_t)cnn::total_params(); }

lbm_status lbm_cnn_create(lbm_cnn** out, int nx, int ny, int nz, const float* init_weights, void* cuda_stream) {
    if (!out || nx < 1 || ny < 1 || nz < 1) return LBM_ERR_ARG;
    *out = nullptr;
    const double P = (double)nx * ny * nz;
    if (P > 268435456.0) return LBM_ERR_ARG;  // 2^28 voxels
    lbm_cnn* c = new (std::nothrow) lbm_cnn();
    if (!c) return LBM_ERR_OOM;
    lbm_alloc_fn a;
    lbm_free_fn r;
    void* u;
    lbm_internal_get_allocator(&a, &r, &u);
    c->alloc = a;
    c->release = r;
    c->user = u;
    c->s.nx = nx;
    c->s.ny = ny;
    c->s.nz = nz;
    c->s.P = (long)nx * ny * nz;
    c->stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return LBM_ERR_CUDA;
    }
    c->wg_blocks = c->nsm;
    c->geom = make_geom(nx, ny, nz);
    const size_t NP = lbm_cnn_param_count();
    const size_t Pn = (size_t)c->s.P;
    bool ok = true;
    auto A = [&](size_t bytes) {
        void* p = cnn_alloc(c, bytes);
        ok = ok && p;
        return p;
    };
    c->master = (float*)A(NP * 4);
    c->grad = (float*)A(NP * 4);
    c->adam_m = (float*)A(NP * 4);
    c->adam_v = (float*)A(NP * 4);
    size_t maxw = 0;
    for (int l = 0; l < cnn::NL; ++l) {
        const size_t w = (size_t)27 * cnn::CH[l] * cnn::CH[l + 1];
        c->wf[l] = (__nv_bfloat16*)A(w * 2);
        c->wb[l] = (__nv_bfloat16*)A(w * 2);
        c->bias[l] = (float*)A((size_t)cnn::CH[l + 1] * 4);
        c->gpad[l] = (float*)A((w + cnn::CH[l + 1]) * 4);
        maxw = std::max(maxw, w + (size_t)cnn::CH[l + 1]);
        c->act[l] = (__nv_bfloat16*)A(Pn * cnn::CH[l] * 2);
    }
    c->partial = (float*)A((size_t)c->wg_blocks * maxw * 4);
    c->out = (float*)A(Pn * 4 * 4);
    c->dA[0] = (__nv_bfloat16*)A(Pn * 32 * 2);
    c->dA[1] = (__nv_bfloat16*)A(Pn * 32 * 2);
    c->dY4 = (__nv_bfloat16*)A(Pn * 16 * 2);
    c->rho_d = (double*)A(Pn * 8);
    c->u_d = (double*)A(3 * Pn * 8);
    c->lpart = (double*)A(((Pn + 255) / 256) * 8);
    c->lsum = (double*)A(8);
    c->status = (int*)A(256);
    if (!ok) {
        lbm_cnn_destroy(c);
        return LBM_ERR_OOM;
    }
    if (!make_maps(c)) {
        lbm_cnn_destroy(c);
        return LBM_ERR_CUDA;
    }
    cudaError_t e = cudaSuccess;
    if (init_weights) {
        e = cudaMemcpyAsync(c->master, init_weights, NP * 4, cudaMemcpyDefault, c->stream);
    } else {
        // He-uniform initialisation from a fixed LCG (deterministic)
        std::vector<float> w(NP);
        unsigned long long st = 0x9E3779B97F4A7C15ull;
        size_t o = 0;
        for (int l = 0; l < cnn::NL; ++l) {
            const int fan_in = 27 * cnn::CH_REAL[l];
            const float lim = std::sqrt(6.0f / fan_in);
            const int nw = 27 * cnn::CH_REAL[l] * cnn::CH_REAL[l + 1];
            for (int i = 0; i < nw; ++i) {
                st = st * 6364136223846793005ull + 1442695040888963407ull;
                const float r01 = (float)((st >> 40) & 0xFFFFFF) / 16777216.0f;
                w[o + i] = (2.f * r01 - 1.f) * lim;
            }
            for (int i = 0; i < cnn::CH_REAL[l + 1]; ++i) w[o + nw + i] = 0.f;
            o += (size_t)cnn::layer_params(l);
        }
        e = cudaMemcpyAsync(c->master, w.data(), NP * 4, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, 256, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dY4, 0, Pn * 16 * 2, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->adam_m, 0, NP * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->adam_v, 0, NP * 4, c->stream);
    for (int l = 0; l < cnn::NL && e == cudaSuccess; ++l)
        e = cudaMemsetAsync(c->act[l], 0, Pn * cnn::CH[l] * 2, c->stream);
    if (e == cudaSuccess) e = pack_all(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        lbm_cnn_destroy(c);
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    *out = c;
    return LBM_OK;
}

void lbm_cnn_destroy(lbm_cnn* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    void* ptrs[] = {c->master, c->grad, c->adam_m, c->adam_v, c->partial, c->out,  c->dA[0],
                    c->dA[1],  c->dY4,  c->rho_d, c->u_d,  c->lpart,  c->lsum, c->status};
    for (void* p : ptrs) cnn_free(c, p);
    for (int l = 0; l < cnn::NL; ++l) {
        cnn_free(c, c->wf[l]);
        cnn_free(c, c->wb[l]);
        cnn_free(c, c->bias[l]);
        cnn_free(c, c->gpad[l]);
        cnn_free(c, c->act[l]);
    }
    delete c;
}

const char* lbm_cnn_last_error(const lbm_cnn* c) { return c ? c->err.c_str() : "null network"; }

lbm_status lbm_cnn_set_weights(lbm_cnn* c, const float* w, size_t count) {
    if (!c || !w || count != lbm_cnn_param_count()) return LBM_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(c->master, w, count * 4, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = pack_all(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? LBM_OK : cnn_cuda_fail(c, e, "lbm_cnn_set_weights");
}

lbm_status lbm_cnn_get_weights(lbm_cnn* c, float* w, size_t count) {
    if (!c || !w || count != lbm_cnn_param_count()) return LBM_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(w, c->master, count * 4, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? LBM_OK : cnn_cuda_fail(c, e, "lbm_cnn_get_weights");
}

lbm_status lbm_cnn_set_input(lbm_cnn* c, double reynolds) {
    if (!c) return LBM_ERR_ARG;
    const long blocks = (c->s.P + 255) / 256;
    cnn::features<<<(unsigned)blocks, 256, 0, c->stream>>>(c->act[0], c->s, (float)((reynolds - 550.0) / 450.0));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : cnn_cuda_fail(c, e, "lbm_cnn_set_input");
}

lbm_status lbm_cnn_set_input_raw(lbm_cnn* c, const float* x, size_t count) {
    // x: [P][16] FP32 input channels (host or device), stored as BF16 [P][16]
    if (!c || !x || count != (size_t)c->s.P * cnn::C_IN_REAL) return LBM_ERR_ARG;
    std::vector<float> h((size_t)c->s.P * 16, 0.f);
    std::vector<float> in(count);
    cudaError_t e = cudaMemcpy(in.data(), x, count * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) return cnn_cuda_fail(c, e, "lbm_cnn_set_input_raw");
    std::vector<__nv_bfloat16> hb((size_t)c->s.P * 16);
    for (long p = 0; p < c->s.P; ++p)
        for (int k = 0; k < 16; ++k)  // channel-chunked layout [2][P][8]
            hb[((size_t)(k / 8) * c->s.P + p) * 8 + k % 8] = __float2bfloat16_rn(in[p * cnn::C_IN_REAL + k]);
    e = cudaMemcpyAsync(c->act[0], hb.data(), hb.size() * 2, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? LBM_OK : cnn_cuda_fail(c, e, "lbm_cnn_set_input_raw");
}

lbm_status lbm_cnn_forward(lbm_cnn* c, float* out, size_t count) {
    // out (optional): [P][4] FP32 prediction (host or device)
    if (!c) return LBM_ERR_ARG;
    if (out && count != (size_t)c->s.P * cnn::C_OUT_REAL) return LBM_ERR_ARG;
    cudaError_t e = forward(c);
    if (e == cudaSuccess && out)
        e = cudaMemcpyAsync(out, c->out, (size_t)c->s.P * 4 * sizeof(float), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? check_status(c, "lbm_cnn_forward") : cnn_cuda_fail(c, e, "lbm_cnn_forward");
}

lbm_status lbm_cnn_gradient(lbm_cnn* c, const double* rho, const double* u, double* loss_out, float* grad_out,
                            size_t count) {
    if (!c || !rho || !u) return LBM_ERR_ARG;
    if (grad_out && count != lbm_cnn_param_count()) return LBM_ERR_ARG;
    cudaError_t e = stage_fields(c, rho, u);
    if (e == cudaSuccess) e = forward(c);
    if (e == cudaSuccess) e = loss(c, rho, u, c->dY4);
    if (e == cudaSuccess) e = backward(c, c->dY4);
    double l = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, c->lsum, 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, c->grad, count * 4, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cnn_cuda_fail(c, e, "lbm_cnn_gradient");
    const lbm_status st = check_status(c, "lbm_cnn_gradient");
    if (st != LBM_OK) return st;
    if (loss_out) *loss_out = l / (4.0 * (double)c->s.P);
    return LBM_OK;
}

lbm_status lbm_cnn_train_step(lbm_cnn* c, const double* rho, const double* u, float lr, double* loss_out) {
    lbm_status st = lbm_cnn_gradient(c, rho, u, loss_out, nullptr, 0);
    if (st != LBM_OK) return st;
    const int n = (int)lbm_cnn_param_count();
    c->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - std::pow(b1, (float)c->adam_t)), c2 = 1.f / (1.f - std::pow(b2, (float)c->adam_t));
    cnn::adam_kernel<<<(n + 255) / 256, 256, 0, c->stream>>>(c->master, c->adam_m, c->adam_v, c->grad, n, lr, b1, b2,
                                                              1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = pack_all(c);
    return e == cudaSuccess ? LBM_OK : cnn_cuda_fail(c, e, "lbm_cnn_train_step");
}

lbm_status lbm_cnn_warm_start(lbm_cnn* c, lbm_ctx* ctx, double reynolds) {
    if (!c || !ctx) return LBM_ERR_ARG;
    lbm_status st = lbm_cnn_set_input(c, reynolds);
    if (st != LBM_OK) return st;
    cudaError_t e = forward(c);
    const long blocks = (c->s.P + 255) / 256;
    if (e == cudaSuccess) {
        cnn::to_fields<<<(unsigned)blocks, 256, 0, c->stream>>>(c->out, c->rho_d, c->u_d, c->s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cnn_cuda_fail(c, e, "lbm_cnn_warm_start");
    st = check_status(c, "lbm_cnn_warm_start");
    if (st != LBM_OK) return st;
    return lbm_init_fields(ctx, c->rho_d, c->u_d, nullptr, nullptr);
}

}  // extern "C"
