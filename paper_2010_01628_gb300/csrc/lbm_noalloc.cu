// lbm_noalloc.cu -- an allocation-free variant of the FP64 mass/momentum
// reduction, for callers that may not allocate device memory.
//
// Who needs it: applications that own every byte of device memory through
// their own pool and forbid side allocations by plug-ins; latency-critical
// loops where cudaMalloc/cudaFree would stall (cudaFree synchronises the
// device); code that runs inside an allocator callback or a memory-pressure
// handler, where calling back into an allocator is not allowed.
//
// The reduction's scratch (one FP64 partial per block) lives in a file-scope
// __device__ array of fixed size.  Every GPU that loads this library holds
// that array (77,824 bytes) until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "lbm_internal.h"
#include "lbm_reduce.cuh"

namespace {

constexpr int NOALLOC_BLOCKS = lbm::RED_BLOCKS;  // fixed grid: 1216 blocks
constexpr int NOALLOC_PARTIALS = NOALLOC_BLOCKS * lbm::RED_WIDTH;
constexpr int MAX_DEVICES = 64;

// Shared by every call on a device: each call's blocks overwrite all of it
// before the final sum reads it, so nothing has to be cleared between calls;
// two calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_PARTIALS];

std::mutex g_setup_mu;
double* g_partials_addr[MAX_DEVICES] = {nullptr};

template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(lbm::RED_THREADS)
    noalloc_reduce_kernel(const S* __restrict__ src, lbm::Box b, double gx, double gy, double gz, double lx, double ly,
                          double lz, double* __restrict__ partials) {
    using namespace lbm;
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
            gather19<S, C, WALLS>(src, b, q, x, y, z, self, (C)lx, (C)ly, (C)lz, f);
            const Moments<C> m = moments19(f);
            const C rho = (C)1 + m.drho;
            // rho u = sum f c + F/2 with F = rho g
            const C px = m.jx + (C)0.5 * rho * (C)gx;
            const C py = m.jy + (C)0.5 * rho * (C)gy;
            const C pz = m.jz + (C)0.5 * rho * (C)gz;
            if (!(rho > (C)0) || !isfinite((double)rho) || !isfinite((double)px) || !isfinite((double)py) ||
                !isfinite((double)pz)) {
                acc.v[6] += 1.0;
            } else {
                acc.v[0] += (double)rho;
                acc.v[1] += (double)px;
                acc.v[2] += (double)py;
                acc.v[3] += (double)pz;
            }
        }
    }
    block_reduce_store(acc, partials);
}

// Fixed-order sum of the partials into out[0..4] (one block, deterministic).
__global__ void noalloc_finalize_kernel(const double* __restrict__ partials, double* __restrict__ out) {
    __shared__ double sh[lbm::RED_THREADS][5];
    double a[5] = {0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < NOALLOC_BLOCKS; i += blockDim.x) {
        a[0] += partials[(size_t)i * lbm::RED_WIDTH + 0];
        a[1] += partials[(size_t)i * lbm::RED_WIDTH + 1];
        a[2] += partials[(size_t)i * lbm::RED_WIDTH + 2];
        a[3] += partials[(size_t)i * lbm::RED_WIDTH + 3];
        a[4] += partials[(size_t)i * lbm::RED_WIDTH + 6];
    }
    for (int k = 0; k < 5; ++k) sh[threadIdx.x][k] = a[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 5; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = sh[0][threadIdx.x];
}

lbm_status set_err(char* err, size_t len, lbm_status s, const char* msg) {
    if (err && len) {
        std::strncpy(err, msg, len - 1);
        err[len - 1] = '\0';
    }
    return s;
}

// Device address of the scratch array for the current device, looked up once
// per device (host code must not use the symbol's host-side name as a
// device pointer).
cudaError_t partials_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = (double*)p;
    }
    *out = g_partials_addr[dev];
    return cudaSuccess;
}

template <typename S, typename C>
cudaError_t launch(const void* pop, const lbm::Box& b, const double* g, const double* lid, double* partials,
                   double* out, cudaStream_t st) {
    const bool walls = (b.periodic & 7u) != 7u;
    if (walls)
        noalloc_reduce_kernel<S, C, true><<<NOALLOC_BLOCKS, lbm::RED_THREADS, 0, st>>>(
            (const S*)pop, b, g[0], g[1], g[2], lid[0], lid[1], lid[2], partials);
    else
        noalloc_reduce_kernel<S, C, false><<<NOALLOC_BLOCKS, lbm::RED_THREADS, 0, st>>>(
            (const S*)pop, b, g[0], g[1], g[2], lid[0], lid[1], lid[2], partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    noalloc_finalize_kernel<<<1, lbm::RED_THREADS, 0, st>>>(partials, out);
    return cudaGetLastError();
}

}  // namespace

extern "C" lbm_status lbm_reduce_state_noalloc(const void* populations, lbm_precision precision, const lbm_grid* grid,
                                               const lbm_forcing* forcing, double* out, void* cuda_stream, char* err,
                                               size_t err_len) {
    if (!populations || !grid || !out) return set_err(err, err_len, LBM_ERR_ARG, "null populations, grid or out");
    if ((int)precision < 0 || (int)precision > 3) return set_err(err, err_len, LBM_ERR_ARG, "unknown precision");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1)
        return set_err(err, err_len, LBM_ERR_ARG, "grid sizes must be >= 1");
    if (grid->ny > 65535 || grid->nz > 65535)
        return set_err(err, err_len, LBM_ERR_ARG, "ny and nz are limited to 65535");
    if (grid->wall_model != LBM_WALL_BOUNCE_BACK)
        return set_err(err, err_len, LBM_ERR_UNSUPPORTED, "only half-way bounce-back walls are supported here");
    if (forcing && forcing->rho_ref != 0.0)
        return set_err(err, err_len, LBM_ERR_UNSUPPORTED, "rho_ref != 0 is supported by the two-phase modules only");
    const double cells = (double)grid->nx * grid->ny * grid->nz;
    if (cells > 2147483647.0)
        return set_err(err, err_len, LBM_ERR_ARG, "grid exceeds the maximum of 2^31 - 1 nodes");
    // Both buffers must be device memory of the current device: a host
    // pointer here would become a faulting (or silently wrong) device access.
    // The query allocates nothing.
    int cur_dev = 0;
    cudaError_t e = cudaGetDevice(&cur_dev);
    if (e != cudaSuccess) return set_err(err, err_len, LBM_ERR_CUDA, "cudaGetDevice failed");
    const void* bufs[2] = {populations, out};
    for (int k = 0; k < 2; ++k) {
        cudaPointerAttributes attr;
        std::memset(&attr, 0, sizeof(attr));
        e = cudaPointerGetAttributes(&attr, bufs[k]);
        if (e != cudaSuccess) {
            cudaGetLastError();  // the failed query leaves a (non-sticky) error behind
            return set_err(err, err_len, LBM_ERR_ARG,
                           k ? "out is not a device pointer" : "populations is not a device pointer");
        }
        const bool on_device = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
        if (!on_device || attr.device != cur_dev)
            return set_err(err, err_len, LBM_ERR_ARG,
                           k ? "out must be device memory of the current device"
                             : "populations must be device memory of the current device");
    }
    double* partials = nullptr;
    e = partials_address(&partials);
    if (e != cudaSuccess) {
        char buf[256];
        std::snprintf(buf, sizeof(buf), "scratch set-up (cudaGetSymbolAddress) failed: %s", cudaGetErrorString(e));
        return set_err(err, err_len, LBM_ERR_CUDA, buf);
    }
    lbm::Box b;
    b.nx = grid->nx;
    b.ny = grid->ny;
    b.nz = grid->nz;
    b.periodic = grid->periodic_mask & 7u;
    b.n = (size_t)grid->nx * grid->ny * grid->nz;
    const double zero[3] = {0.0, 0.0, 0.0};
    const double* g = forcing ? forcing->g : zero;
    const double lid[3] = {(b.periodic & 2u) ? 0.0 : grid->lid_u[0], (b.periodic & 2u) ? 0.0 : grid->lid_u[1],
                           (b.periodic & 2u) ? 0.0 : grid->lid_u[2]};
    cudaStream_t st = (cudaStream_t)cuda_stream;
    switch (precision) {
        case LBM_FP64: e = launch<double, double>(populations, b, g, lid, partials, out, st); break;
        case LBM_FP32: e = launch<float, float>(populations, b, g, lid, partials, out, st); break;
        case LBM_FP16_SHIFTED: e = launch<__half, float>(populations, b, g, lid, partials, out, st); break;
        case LBM_BF16_SHIFTED: e = launch<__nv_bfloat16, float>(populations, b, g, lid, partials, out, st); break;
    }
    if (e != cudaSuccess) {
        char buf[256];
        std::snprintf(buf, sizeof(buf), "launch failed: %s", cudaGetErrorString(e));
        return set_err(err, err_len, LBM_ERR_CUDA, buf);
    }
    return set_err(err, err_len, LBM_OK, "");
}
