// lbm_batch.cu -- batched parameter sweeps: many independent domains of
// uneven sizes advanced by ONE persistent cooperative kernel per call to
// lbm_batch_step (n steps inside the kernel, a grid-wide barrier between
// steps), replayed from a captured CUDA graph.
//
// Work decomposition: every domain is cut into tiles of `threads` consecutive
// nodes (x fastest); tiles of all domains form one global index space that the
// resident CTAs walk with a grid stride.  A CTA finds its tile's domain by a
// binary search over the per-domain first-tile table (uniform across the CTA).
// Per-domain parameters (size, boundaries, omega, g, Hartmann field, colour
// densities and surface tension, Shan-Chen interaction strength...) come from
// a small device table.  The colour-gradient and Shan-Chen steps take two
// passes (order parameter or pseudopotential, then collision), so their
// kernels run a grid-wide barrier after each pass.
//
// The barrier waits are bounded: a CTA that waits longer than the timeout
// records LBM_ERR_TIMEOUT and every CTA returns; the host reads the status at
// the next lbm_sync.  The buffers are rewritten between barriers, so the
// read-only (.nc) path is not valid here: the kernel uses plain cached loads,
// which the barrier's GPU-scope fences order after the other CTAs' stores.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_cgm.cuh"
#include "lbm_fluid.cuh"
#include "lbm_internal.h"
#include "lbm_mhd.cuh"
#include "lbm_sc.cuh"

namespace lbm {

struct BatchDomain {
    FluidArgs fl;     // box, omega, g, lid
    MhdArgs mh;       // box, omega, tau_m, g, b_wall
    CgmArgs cg;       // box, omega, alpha_r, alpha_b, A, beta, g, rho_ref g
    ScArgs sc;        // box, omega, G, g, rho_ref g, lid
    size_t off;       // element offset of the domain's plane 0 in a state copy
    size_t soff;      // offset of the domain's node 0 in each scratch plane (colour gradient)
    uint32_t tile0;   // first global tile of the domain
    uint32_t ntiles;
};

struct BarrierState {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

constexpr unsigned long long BARRIER_TIMEOUT_NS = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sense-counting grid barrier with a bounded wait.  `expected` is the number
// of CTAs that must arrive.  Returns false (and every CTA should return) if the
// wait timed out here or an error was raised elsewhere.
__device__ bool grid_barrier(BarrierState* bs, unsigned expected, unsigned long long timeout_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &bs->gen;
        volatile int* verr = &bs->err;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&bs->count, 1u) + 1u;
        int res = 1;
        if (arrived == expected) {
            atomicExch(&bs->count, 0u);
            __threadfence();
            atomicAdd(&bs->gen, 1u);
        } else {
            const unsigned long long t0 = globaltimer_ns();
            while (*vgen == g) {
                if (*verr != 0) {
                    res = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > timeout_ns) {
                    atomicCAS(&bs->err, 0, (int)LBM_ERR_TIMEOUT);
                    res = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok = res;
    }
    __syncthreads();
    return ok != 0;
}

// Domain of global tile t (binary search over the first-tile table; uniform
// across the CTA) and the node's coordinates; false past the domain's end.
__device__ __forceinline__ bool tile_node(const BatchDomain* __restrict__ doms, int nd, uint32_t t, int& d, int& x,
                                          int& y, int& z) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (doms[mid].tile0 <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    d = lo;
    const Box& b = doms[lo].fl.box;
    const uint32_t cell = (t - doms[lo].tile0) * blockDim.x + threadIdx.x;
    if (cell >= (uint32_t)b.n) return false;
    const uint32_t plane = (uint32_t)b.nx * (uint32_t)b.ny;
    const uint32_t zz = cell / plane;
    const uint32_t r = cell - zz * plane;
    const uint32_t yy = r / (uint32_t)b.nx;
    x = (int)(r - yy * (uint32_t)b.nx);
    y = (int)yy;
    z = (int)zz;
    return true;
}

// scratch (colour gradient only): phi of every domain's nodes, then rho_r,
// each `scratch_n` values long; a domain's nodes start at its soff.  WALLS:
// false when every domain is periodic in all three directions (the node code
// then carries no bounce-back).  The FP32 colour-gradient and Shan-Chen
// variants are held to 64 registers (4 CTAs of 256 or 8 of 128 per SM): their
// first passes wait on the neighbours' loads and need the warps.  Measured on
// the 64-domain sweeps: Shan-Chen 20.6 GLUPS at 64 registers, 19.0 at 96 and
// 18.9 at 48; colour gradient 14.0 at 64, 13.7 at 80 and 12.3 at 48.
template <int PHYS, typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(256, ((PHYS == LBM_PHYS_CGM || PHYS == LBM_PHYS_SC) && sizeof(S) == 4) ? 4 : 1)
    batch_kernel(S* bufA, S* bufB, const BatchDomain* __restrict__ doms, int nd,
                                                    uint32_t ntiles, long nsteps, int parity0, int dry,
                                                    BarrierState* bs, unsigned long long timeout_ns, C* scratch,
                                                    size_t scratch_n) {
    for (long s = 0; s < nsteps; ++s) {
        const int par = dry ? parity0 : (int)((parity0 + s) & 1);
        const S* src = par ? bufB : bufA;
        S* dst = par ? bufA : bufB;
        if (PHYS == LBM_PHYS_SC) {
            // pass 1: pseudopotential psi = 1 - exp(-rho) of every node
            for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
                int d, x, y, z;
                if (tile_node(doms, nd, t, d, x, y, z)) {
                    const BatchDomain& D = doms[d];
                    sc_psi_node<S, C, WALLS, false>(src + D.off, scratch + D.soff, D.sc, x, y, z);
                }
            }
            if (!grid_barrier(bs, gridDim.x, timeout_ns)) return;
            // pass 2: force, forced collision
            for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
                int d, x, y, z;
                if (tile_node(doms, nd, t, d, x, y, z)) {
                    const BatchDomain& D = doms[d];
                    sc_collide_node<S, C, WALLS, false>(src + D.off, dst + D.off, scratch + D.soff, D.sc, x, y, z);
                }
            }
        } else if (PHYS == LBM_PHYS_CGM) {
            // pass 1: order parameter and red density of every node
            for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
                int d, x, y, z;
                if (tile_node(doms, nd, t, d, x, y, z)) {
                    const BatchDomain& D = doms[d];
                    cgm_phi_node<S, C, WALLS, false>(src + D.off, scratch + D.soff, scratch + scratch_n + D.soff, D.cg,
                                                    x, y, z);
                }
            }
            if (!grid_barrier(bs, gridDim.x, timeout_ns)) return;
            // pass 2: collision, perturbation, recolouring
            for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
                int d, x, y, z;
                if (tile_node(doms, nd, t, d, x, y, z)) {
                    const BatchDomain& D = doms[d];
                    cgm_collide_node<S, C, WALLS, false>(src + D.off, dst + D.off, scratch + D.soff,
                                                        scratch + scratch_n + D.soff, D.cg, x, y, z);
                }
            }
        } else {
            for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
                int d, x, y, z;
                if (tile_node(doms, nd, t, d, x, y, z)) {
                    const BatchDomain& D = doms[d];
                    if (PHYS == LBM_PHYS_MHD)
                        mhd_node<S, C, WALLS, false>(src + D.off, dst + D.off, D.mh, x, y, z);
                    else
                        fluid_node<S, C, WALLS, false>(src + D.off, dst + D.off, D.fl, x, y, z);
                }
            }
        }
        if (s + 1 < nsteps && !grid_barrier(bs, gridDim.x, timeout_ns)) return;
    }
}

// Diagnostic: a barrier that waits for one CTA more than the grid has, so
// every wait runs into its (short) limit; used to check that bounded waits
// end and report LBM_ERR_TIMEOUT.
__global__ void barrier_selftest_kernel(BarrierState* bs, unsigned long long timeout_ns) {
    grid_barrier(bs, gridDim.x + 1, timeout_ns);
}

}  // namespace lbm

using lbm::BarrierState;
using lbm::BatchDomain;

struct BatchState {
    int nd = 0;
    std::vector<lbm_ctx*> views;
    std::vector<BatchDomain> doms;
    BatchDomain* d_doms = nullptr;
    BarrierState* d_bar = nullptr;
    uint32_t ntiles = 0;
    int threads = 256;
    int ctas_per_sm = 0;  // 0 = as many as fit
    int grid = 0;
    int sms = 0;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long graph_n[2] = {-1, -1};
    bool graph_ok = true;
    size_t state_elems = 0;
    size_t scratch_n = 0;  // values per scratch plane (colour gradient: all domains' nodes)
    bool walls = true;     // false: every domain periodic in x, y and z
    unsigned long long timeout_ns = lbm::BARRIER_TIMEOUT_NS;
};

namespace {

template <int PHYS, typename S, typename C>
void* kernel_ptr(bool walls) {
    return walls ? (void*)lbm::batch_kernel<PHYS, S, C, true> : (void*)lbm::batch_kernel<PHYS, S, C, false>;
}

void* batch_kernel_for(const lbm_ctx* c) {
    const bool f64 = c->prec == LBM_FP64, w = c->batch->walls;
    switch (c->physics) {
        case LBM_PHYS_MHD:
            return f64 ? kernel_ptr<LBM_PHYS_MHD, double, double>(w) : kernel_ptr<LBM_PHYS_MHD, float, float>(w);
        case LBM_PHYS_CGM:
            return f64 ? kernel_ptr<LBM_PHYS_CGM, double, double>(w) : kernel_ptr<LBM_PHYS_CGM, float, float>(w);
        case LBM_PHYS_SC:
            return f64 ? kernel_ptr<LBM_PHYS_SC, double, double>(w) : kernel_ptr<LBM_PHYS_SC, float, float>(w);
        default:
            return f64 ? kernel_ptr<0, double, double>(w) : kernel_ptr<0, float, float>(w);
    }
}

void build_tiles(BatchState* B) {
    uint32_t t = 0;
    for (auto& d : B->doms) {
        d.tile0 = t;
        d.ntiles = (uint32_t)((d.fl.box.n + B->threads - 1) / B->threads);
        t += d.ntiles;
    }
    B->ntiles = t;
}

cudaError_t configure(lbm_ctx* c) {
    BatchState* B = c->batch;
    build_tiles(B);
    cudaError_t e = cudaMemcpyAsync(B->d_doms, B->doms.data(), sizeof(BatchDomain) * B->nd, cudaMemcpyHostToDevice,
                                    c->stream);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_for(c), B->threads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int want = B->ctas_per_sm > 0 ? std::min(B->ctas_per_sm, per_sm) : per_sm;
    long grid = (long)want * B->sms;
    if (grid > (long)B->ntiles) grid = B->ntiles;
    B->grid = (int)std::max(1L, grid);
    for (int k = 0; k < 2; ++k) {
        if (B->graph[k]) cudaGraphExecDestroy(B->graph[k]);
        B->graph[k] = nullptr;
        B->graph_n[k] = -1;
    }
    return cudaStreamSynchronize(c->stream);
}

cudaError_t launch_direct(lbm_ctx* c, cudaStream_t st, long n, int parity, int dry) {
    BatchState* B = c->batch;
    cudaError_t e = cudaMemsetAsync(B->d_bar, 0, sizeof(BarrierState), st);
    if (e != cudaSuccess) return e;
    void* a = c->buf[0];
    void* b = c->buf[1];
    BatchDomain* doms = B->d_doms;
    int nd = B->nd;
    uint32_t nt = B->ntiles;
    BarrierState* bar = B->d_bar;
    unsigned long long to = B->timeout_ns;
    void* scratch = c->phi;  // colour gradient: phi and rho_r planes of all domains (else unused)
    size_t scratch_n = B->scratch_n;
    void* args[] = {&a, &b, &doms, &nd, &nt, &n, &parity, &dry, &bar, &to, &scratch, &scratch_n};
    return cudaLaunchCooperativeKernel(batch_kernel_for(c), dim3(B->grid), dim3(B->threads), args, 0, st);
}

// Capture (once per starting parity and step count) and replay.
cudaError_t run_batch(lbm_ctx* c, long n, int dry) {
    BatchState* B = c->batch;
    const int parity = c->cur;
    cudaError_t e = cudaEventRecord(B->ev_in, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->cap, B->ev_in, 0);
    if (e != cudaSuccess) return e;
    if (dry || !B->graph_ok) {
        e = launch_direct(c, B->cap, n, parity, dry);
    } else {
        if (!B->graph[parity] || B->graph_n[parity] != n) {
            if (B->graph[parity]) cudaGraphExecDestroy(B->graph[parity]);
            B->graph[parity] = nullptr;
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t el = launch_direct(c, B->cap, n, parity, 0);
                e = cudaStreamEndCapture(B->cap, &g);
                if (e == cudaSuccess) e = el;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph[parity], g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                // capture of cooperative launches unavailable: launch directly from now on
                cudaGetLastError();
                B->graph_ok = false;
                B->graph[parity] = nullptr;
                e = launch_direct(c, B->cap, n, parity, 0);
            } else {
                B->graph_n[parity] = n;
            }
        }
        if (B->graph_ok && B->graph[parity]) e = cudaGraphLaunch(B->graph[parity], B->cap);
    }
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(B->ev_out, B->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, B->ev_out, 0);
    if (e == cudaSuccess && !dry && (n & 1)) {
        c->cur ^= 1;
        for (lbm_ctx* v : B->views) v->cur = c->cur;
    }
    return e;
}

}  // namespace

namespace lbm {

// Timed dry run of the persistent kernel (state unchanged) for the autotuner.
cudaError_t batch_time_config(lbm_ctx* c, int threads, int ctas_per_sm, long steps, float* ms) {
    BatchState* B = c->batch;
    B->threads = threads;
    B->ctas_per_sm = ctas_per_sm;
    cudaError_t e = configure(c);
    if (e != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    e = run_batch(c, 2, 1);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(a, c->stream);
    if (e == cudaSuccess) e = run_batch(c, steps, 1);
    if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

cudaError_t batch_apply_config(lbm_ctx* c, int threads, int ctas_per_sm) {
    c->batch->threads = threads;
    c->batch->ctas_per_sm = ctas_per_sm;
    return configure(c);
}

void batch_destroy(lbm_ctx* c) {
    BatchState* B = c->batch;
    if (!B) return;
    for (int k = 0; k < 2; ++k)
        if (B->graph[k]) cudaGraphExecDestroy(B->graph[k]);
    if (B->ev_in) cudaEventDestroy(B->ev_in);
    if (B->ev_out) cudaEventDestroy(B->ev_out);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (lbm_ctx* v : B->views) delete v;
    delete B;
    c->batch = nullptr;
}

}  // namespace lbm

// ---------------------------------------------------------------------------
extern "C" {

lbm_status lbm_batch_create(lbm_ctx** out, int ndomains, const lbm_grid* grids, const lbm_relax* relax,
                            const lbm_forcing* forcing, lbm_physics physics, const lbm_physparams* phys,
                            lbm_precision precision, void* cuda_stream) {
    if (!out || ndomains < 1 || !grids || !relax) return LBM_ERR_ARG;
    *out = nullptr;
    if (physics != LBM_PHYS_FLUID && physics != LBM_PHYS_MHD && physics != LBM_PHYS_CGM && physics != LBM_PHYS_SC)
        return LBM_ERR_UNSUPPORTED;
    if (precision != LBM_FP32 && precision != LBM_FP64) return LBM_ERR_UNSUPPORTED;
    if ((physics == LBM_PHYS_MHD || physics == LBM_PHYS_CGM || physics == LBM_PHYS_SC) && !phys) return LBM_ERR_ARG;
    const int planes = physics == LBM_PHYS_MHD ? 40 : (physics == LBM_PHYS_CGM ? 24 : 19);
    const size_t elem = precision == LBM_FP64 ? 8 : 4;
    size_t total = 0, max_plane = 0, cells = 0;
    for (int d = 0; d < ndomains; ++d) {
        const lbm_grid& g = grids[d];
        if (g.nx < 1 || g.ny < 1 || g.nz < 1) return LBM_ERR_ARG;
        const double n = (double)g.nx * g.ny * g.nz;
        if (n >= 2147483648.0) return LBM_ERR_ARG;
        if (!(relax[d].omega > 0.0 && relax[d].omega < 2.0)) return LBM_ERR_ARG;
        if (relax[d].omega_bulk != 1.0 || relax[d].omega_3 != 1.0 || relax[d].omega_4 != 1.0)
            return LBM_ERR_UNSUPPORTED;
        if (physics == LBM_PHYS_MHD && !(phys[d].tau_m > 0.5)) return LBM_ERR_ARG;
        if (physics == LBM_PHYS_CGM &&
            !(phys[d].alpha_r >= 0.0 && phys[d].alpha_r < 1.0 && phys[d].alpha_b >= 0.0 && phys[d].alpha_b < 1.0))
            return LBM_ERR_ARG;
        if (physics == LBM_PHYS_SC && !std::isfinite(phys[d].G)) return LBM_ERR_ARG;
        if (forcing && forcing[d].rho_ref != 0.0 && physics != LBM_PHYS_CGM && physics != LBM_PHYS_SC)
            return LBM_ERR_UNSUPPORTED;
        if (g.wall_model != LBM_WALL_BOUNCE_BACK || relax[d].moment_space != LBM_MOMENTS_CENTRAL)
            return LBM_ERR_UNSUPPORTED;
        if ((physics == LBM_PHYS_MHD || physics == LBM_PHYS_CGM) && (g.periodic_mask & 2u) == 0 &&
            (g.lid_u[0] != 0.0 || g.lid_u[1] != 0.0 || g.lid_u[2] != 0.0))
            return LBM_ERR_UNSUPPORTED;
        const size_t nn = (size_t)g.nx * g.ny * g.nz;
        total += ((size_t)planes * nn + 63) / 64 * 64;  // each domain block starts 256-byte aligned
        max_plane = std::max(max_plane, (size_t)g.nx * g.ny);
        cells += nn;
    }
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    BatchState* B = new (std::nothrow) BatchState();
    if (!c || !B) {
        delete c;
        delete B;
        return LBM_ERR_OOM;
    }
    c->batch = B;
    c->owns = true;
    c->grid = grids[0];
    c->relax = relax[0];
    if (forcing) c->forcing = forcing[0];
    c->physics = physics;
    if (phys) c->phys = phys[0];
    c->prec = precision;
    c->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);
    c->elem = elem;
    c->planes = planes;
    c->box.nx = c->box.ny = c->box.nz = 0;
    c->box.n = cells;
    B->nd = ndomains;
    lbm_status st = lbm_internal_alloc_batch(c, total, cells, max_plane);
    if (st != LBM_OK) {
        lbm::batch_destroy(c);
        lbm_internal_release(c);
        delete c;
        return st;
    }
    B->state_elems = total;
    B->scratch_n = cells;
    B->walls = false;
    for (int d = 0; d < ndomains; ++d) B->walls = B->walls || (grids[d].periodic_mask & 7u) != 7u;
    cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaError_t e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming);
    size_t off = 0, uoff = 0, soff = 0;
    for (int d = 0; d < ndomains && e == cudaSuccess; ++d) {
        const lbm_grid& g = grids[d];
        BatchDomain D;
        std::memset(&D, 0, sizeof(D));
        D.fl.box.nx = g.nx;
        D.fl.box.ny = g.ny;
        D.fl.box.nz = g.nz;
        D.fl.box.periodic = g.periodic_mask & 7u;
        D.fl.box.n = (size_t)g.nx * g.ny * g.nz;
        D.fl.omega = relax[d].omega;
        for (int a = 0; a < 3; ++a) {
            D.fl.g[a] = forcing ? forcing[d].g[a] : 0.0;
            D.fl.lid[a] = (g.periodic_mask & 2u) ? 0.0 : g.lid_u[a];
        }
        D.mh.box = D.fl.box;
        D.mh.omega = relax[d].omega;
        if (physics == LBM_PHYS_MHD) {
            D.mh.tau_m = phys[d].tau_m;
            D.mh.inv_tau_m = 1.0 / phys[d].tau_m;
            D.mh.jfac = 1.0 / (phys[d].tau_m * lbm::CSM2);
            for (int a = 0; a < 3; ++a) {
                D.mh.g[a] = D.fl.g[a];
                D.mh.bw[a] = phys[d].b_wall[a];
            }
        }
        if (physics == LBM_PHYS_CGM) {
            D.cg.box = D.fl.box;
            D.cg.omega = relax[d].omega;
            D.cg.alpha_r = phys[d].alpha_r;
            D.cg.alpha_b = phys[d].alpha_b;
            D.cg.A = phys[d].A;
            D.cg.beta = phys[d].beta;
            for (int a = 0; a < 3; ++a) {
                D.cg.g[a] = D.fl.g[a];
                D.cg.rg[a] = forcing ? forcing[d].rho_ref * forcing[d].g[a] : 0.0;
            }
        }
        if (physics == LBM_PHYS_SC) {
            D.sc.box = D.fl.box;
            D.sc.omega = relax[d].omega;
            D.sc.G = phys[d].G;
            for (int a = 0; a < 3; ++a) {
                D.sc.g[a] = D.fl.g[a];
                D.sc.rg[a] = forcing ? forcing[d].rho_ref * forcing[d].g[a] : 0.0;
                D.sc.lid[a] = D.fl.lid[a];
            }
        }
        D.off = off;
        D.soff = soff;
        B->doms.push_back(D);
        // a view context per domain (init/fields/reduce/populations)
        lbm_ctx* v = new (std::nothrow) lbm_ctx();
        if (!v) {
            e = cudaErrorMemoryAllocation;
            break;
        }
        *v = *c;
        v->batch = nullptr;
        v->owns = false;
        v->parent = c;
        v->grid = g;
        v->relax = relax[d];
        if (forcing) v->forcing = forcing[d];
        else std::memset(&v->forcing, 0, sizeof(v->forcing));
        if (phys) v->phys = phys[d];
        v->box = D.fl.box;
        v->buf[0] = (char*)c->buf[0] + off * elem;
        v->buf[1] = (char*)c->buf[1] + off * elem;
        v->uprev = (char*)c->uprev + uoff * (precision == LBM_FP64 ? 8 : 4);  // compute-type velocities
        v->phi = c->phi ? (char*)c->phi + soff * (precision == LBM_FP64 ? 8 : 4) : nullptr;
        v->block_x = g.nx >= 256 ? 256 : (g.nx >= 128 ? 128 : (g.nx >= 64 ? 64 : 32));
        B->views.push_back(v);
        off += ((size_t)planes * D.fl.box.n + 63) / 64 * 64;
        uoff += 3 * D.fl.box.n;
        soff += D.fl.box.n;
    }
    if (e == cudaSuccess) e = configure(c);
    // rest state for every domain
    for (int d = 0; d < ndomains && e == cudaSuccess; ++d) {
        lbm_ctx* v = B->views[d];
        for (int z0 = 0; z0 < v->box.nz && e == cudaSuccess; ++z0) e = lbm_internal_init_slab(v, z0, 1, true);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        lbm::batch_destroy(c);
        lbm_internal_release(c);
        delete c;
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    *out = c;
    return LBM_OK;
}

lbm_status lbm_batch_domain(lbm_ctx* c, int d, lbm_ctx** view) {
    if (!c || !c->batch || !view || d < 0 || d >= c->batch->nd) return LBM_ERR_ARG;
    c->batch->views[d]->cur = c->cur;
    *view = c->batch->views[d];
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_ctx* c, long n) {
    if (!c || !c->batch || n < 0) return LBM_ERR_ARG;
    if (n == 0) return LBM_OK;
    cudaError_t e = run_batch(c, n, 0);
    if (e != cudaSuccess) {
        c->err = std::string("lbm_batch_step: ") + cudaGetErrorString(e);
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_ctx* c, int* threads, int* grid, int* graph, long* tiles) {
    if (!c || !c->batch) return LBM_ERR_ARG;
    if (threads) *threads = c->batch->threads;
    if (grid) *grid = c->batch->grid;
    if (graph) *graph = c->batch->graph_ok ? 1 : 0;
    if (tiles) *tiles = (long)c->batch->ntiles;
    return LBM_OK;
}

lbm_status lbm_barrier_selftest(double timeout_s, int* observed) {
    if (!observed || !(timeout_s > 0.0) || timeout_s > 10.0) return LBM_ERR_ARG;
    BarrierState* bs = nullptr;
    if (cudaMalloc(&bs, sizeof(BarrierState)) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_OOM;
    }
    cudaError_t e = cudaMemset(bs, 0, sizeof(BarrierState));
    if (e == cudaSuccess) {
        lbm::barrier_selftest_kernel<<<4, 64>>>(bs, (unsigned long long)(timeout_s * 1e9));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    BarrierState h;
    if (e == cudaSuccess) e = cudaMemcpy(&h, bs, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(bs);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    *observed = h.err;
    return LBM_OK;
}

}  // extern "C"

lbm_status lbm_internal_batch_status(lbm_ctx* c) {
    if (!c || !c->batch) return LBM_OK;
    BarrierState h;
    cudaError_t e = cudaMemcpy(&h, c->batch->d_bar, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    if (h.err == (int)LBM_ERR_TIMEOUT) {
        c->err = "batch grid barrier wait exceeded its limit";
        return LBM_ERR_TIMEOUT;
    }
    return LBM_OK;
}

size_t lbm_internal_batch_state_elems(const lbm_ctx* c) { return c->batch ? c->batch->state_elems : 0; }

lbm_status lbm_internal_alloc_batch_tables(lbm_ctx* c) {
    BatchState* B = c->batch;
    B->d_doms = (BatchDomain*)lbm_internal_dev_alloc(c, sizeof(BatchDomain) * (size_t)B->nd);
    B->d_bar = (BarrierState*)lbm_internal_dev_alloc(c, sizeof(BarrierState));
    if (!B->d_doms || !B->d_bar) return LBM_ERR_OOM;
    return LBM_OK;
}

void lbm_internal_free_batch_tables(lbm_ctx* c) {
    BatchState* B = c->batch;
    if (!B) return;
    lbm_internal_dev_free(c, B->d_doms);
    lbm_internal_dev_free(c, B->d_bar);
    B->d_doms = nullptr;
    B->d_bar = nullptr;
}
