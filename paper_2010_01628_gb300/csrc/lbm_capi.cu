// lbm_capi.cu -- the extern "C" entry points of include/lbm.h: context
// life-cycle, field transfer in z-slabs, stepping, reductions and the
// steady-state driver.  All device work is ordered on the context stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "lbm_internal.h"

namespace {

lbm_alloc_fn g_alloc = nullptr;
lbm_free_fn g_release = nullptr;
void* g_user = nullptr;

// Cells per field slab: whole z-planes, about 8M cells (8 FP64 planes = 512 MB).
constexpr size_t SLAB_TARGET_CELLS = size_t(8) << 20;

lbm_status fail(lbm_ctx* c, lbm_status s, const char* fmt, const char* detail = "") {
    if (c) {
        char buf[512];
        std::snprintf(buf, sizeof(buf), fmt, detail);
        c->err = buf;
    }
    return s;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
    if (c) {
        char buf[512];
        std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
        c->err = buf;
    }
    return LBM_ERR_CUDA;
}

void* dev_alloc(lbm_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (c->alloc) return c->alloc(bytes, (void*)c->stream, c->user);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(lbm_ctx* c, void* p) {
    if (!p) return;
    if (c->release)
        c->release(p, (void*)c->stream, c->user);
    else
        cudaFree(p);
}

size_t compute_bytes(const lbm_ctx* c) { return c->prec == LBM_FP64 ? 8 : 4; }

int slab_planes(const lbm_ctx* c) {
    const size_t plane = (size_t)c->box.nx * c->box.ny;
    size_t k = c->staging_cells / (plane ? plane : 1);  // the staging slab decides
    if (k < 1) k = 1;
    if (k > (size_t)c->box.nz) k = (size_t)c->box.nz;
    return (int)k;
}

cudaError_t phys_step(lbm_ctx* c, long n, bool dry = false) {
    if (c->q == 27) return lbm::q27_step(c, n, dry);
    switch (c->physics) {
        case LBM_PHYS_FLUID: return lbm::fluid_step(c, n, dry);
        case LBM_PHYS_MHD: return lbm::mhd_step(c, n, dry);
        case LBM_PHYS_CGM: return lbm::cgm_step(c, n, dry);
        case LBM_PHYS_SC: return lbm::sc_step(c, n, dry);
    }
    return cudaErrorInvalidValue;
}
cudaError_t phys_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform) {
    if (c->q == 27) return lbm::q27_init(c, slab, z0, nzs, uniform);
    switch (c->physics) {
        case LBM_PHYS_FLUID: return lbm::fluid_init(c, slab, z0, nzs, uniform);
        case LBM_PHYS_MHD: return lbm::mhd_init(c, slab, z0, nzs, uniform);
        case LBM_PHYS_CGM: return lbm::cgm_init(c, slab, z0, nzs, uniform);
        case LBM_PHYS_SC: return lbm::fluid_init(c, slab, z0, nzs, uniform);
    }
    return cudaErrorInvalidValue;
}
cudaError_t phys_fields(lbm_ctx* c, double* slab, int z0, int nzs) {
    if (c->q == 27) return lbm::q27_fields(c, slab, z0, nzs);
    switch (c->physics) {
        case LBM_PHYS_FLUID: return lbm::fluid_fields(c, slab, z0, nzs);
        case LBM_PHYS_MHD: return lbm::mhd_fields(c, slab, z0, nzs);
        case LBM_PHYS_CGM: return lbm::cgm_fields(c, slab, z0, nzs);
        case LBM_PHYS_SC: return lbm::sc_fields(c, slab, z0, nzs);
    }
    return cudaErrorInvalidValue;
}
cudaError_t phys_reduce(lbm_ctx* c, bool record) {
    if (c->q == 27) return lbm::q27_reduce(c, record);
    switch (c->physics) {
        case LBM_PHYS_FLUID: return lbm::fluid_reduce(c, record);
        case LBM_PHYS_MHD: return lbm::mhd_reduce(c, record);
        case LBM_PHYS_CGM: return lbm::cgm_reduce(c, record);
        case LBM_PHYS_SC: return lbm::sc_reduce(c, record);
    }
    return cudaErrorInvalidValue;
}

void release_all(lbm_ctx* c) {
    if (!c->owns) return;
    for (int k = 0; k < 2; ++k) dev_free(c, c->buf[k]);
    dev_free(c, c->phi);
    dev_free(c, c->uprev);
    dev_free(c, c->partials);
    dev_free(c, c->result);
    dev_free(c, c->staging);
    dev_free(c, c->status);
    if (c->result_host) cudaFreeHost(c->result_host);
    for (int b = 0; b < 2; ++b) {
        if (c->slab_ready[b]) cudaEventDestroy(c->slab_ready[b]);
        if (c->slab_free[b]) cudaEventDestroy(c->slab_free[b]);
    }
    if (c->fields_start) cudaEventDestroy(c->fields_start);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
}

// The copy stream and the events of the double-buffered field slabs.
bool make_copy_stream(lbm_ctx* c) {
    bool ok = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaEventCreateWithFlags(&c->slab_ready[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->slab_free[b], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->fields_start, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
    return ok;
}

// Field slab b of the two (8 FP64 planes of staging_cells each).
double* slab_buf(lbm_ctx* c, int b) { return c->staging + (size_t)b * 8 * c->staging_cells; }

// Status word of the bounded device waits (TMA-staged kernel); read after a
// synchronisation.
lbm_status device_status(lbm_ctx* c) {
    if (!c->status) return LBM_OK;
    int h = 0;
    if (cudaMemcpy(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ERR_CUDA;
    if (h == (int)LBM_ERR_TIMEOUT) {
        c->err = "a bounded device wait (TMA-staged step) exceeded its limit";
        return LBM_ERR_TIMEOUT;
    }
    return LBM_OK;
}

}  // namespace

void* lbm_internal_dev_alloc(lbm_ctx* c, size_t bytes) { return dev_alloc(c, bytes); }
void lbm_internal_get_allocator(lbm_alloc_fn* a, lbm_free_fn* r, void** user) {
    *a = g_alloc;
    *r = g_release;
    *user = g_user;
}
void lbm_internal_dev_free(lbm_ctx* c, void* p) { dev_free(c, p); }
void lbm_internal_release(lbm_ctx* c) {
    if (c->batch) lbm_internal_free_batch_tables(c);
    release_all(c);
}
cudaError_t lbm_internal_init_slab(lbm_ctx* c, int z0, int nzs, bool uniform) {
    return phys_init(c, c->staging, z0, nzs, uniform);
}
cudaError_t lbm_internal_step(lbm_ctx* c, long n, bool dry) { return phys_step(c, n, dry); }

// Buffers of a batch: two state copies of `state_elems` values, the residual
// velocity of every node, reduction scratch, a staging slab sized for the
// largest domain plane, and the device tables of the persistent kernel.
lbm_status lbm_internal_alloc_batch(lbm_ctx* c, size_t state_elems, size_t cells, size_t max_plane) {
    c->alloc = g_alloc;
    c->release = g_release;
    c->user = g_user;
    const size_t cb = compute_bytes(c);
    size_t k = SLAB_TARGET_CELLS / (max_plane ? max_plane : 1);
    if (k < 1) k = 1;
    c->staging_cells = max_plane * k;
    c->buf[0] = dev_alloc(c, state_elems * c->elem);
    c->buf[1] = dev_alloc(c, state_elems * c->elem);
    c->uprev = dev_alloc(c, 3 * cells * cb);
    c->partials = (double*)dev_alloc(c, sizeof(double) * lbm::RED_WIDTH * lbm::RED_BLOCKS);
    c->result = (double*)dev_alloc(c, sizeof(double) * lbm::RED_WIDTH);
    c->staging = (double*)dev_alloc(c, sizeof(double) * 2 * 8 * c->staging_cells);
    if (!(c->buf[0] && c->buf[1] && c->uprev && c->partials && c->result && c->staging)) return LBM_ERR_OOM;
    if (!make_copy_stream(c)) return LBM_ERR_CUDA;
    // colour gradient: phi and rho_r of every domain's nodes; Shan-Chen: psi;
    // rebuilt each step
    if (c->physics == LBM_PHYS_CGM || c->physics == LBM_PHYS_SC) {
        c->phi = dev_alloc(c, (c->physics == LBM_PHYS_CGM ? 2 : 1) * cells * cb);
        if (!c->phi) return LBM_ERR_OOM;
    }
    if (cudaMallocHost((void**)&c->result_host, sizeof(double) * lbm::RED_WIDTH) != cudaSuccess) {
        cudaGetLastError();
        c->result_host = nullptr;
        return LBM_ERR_OOM;
    }
    return lbm_internal_alloc_batch_tables(c);
}

extern "C" {

const char* lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_ERR_ARG: return "invalid argument";
        case LBM_ERR_OOM: return "device allocation failed";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_DIVERGED: return "simulation diverged";
        case LBM_ERR_TIMEOUT: return "bounded device wait timed out";
        case LBM_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : "null context"; }

lbm_status lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void* user) {
    if ((alloc == nullptr) != (release == nullptr)) return LBM_ERR_ARG;
    g_alloc = alloc;
    g_release = release;
    g_user = user;
    return LBM_OK;
}

lbm_status lbm_create(lbm_ctx** out, const lbm_grid* grid, lbm_lattice lattice, const lbm_relax* relax,
                      const lbm_forcing* forcing, lbm_physics physics, const lbm_physparams* phys,
                      lbm_precision precision, void* cuda_stream) {
    if (!out || !grid || !relax) return LBM_ERR_ARG;
    *out = nullptr;
    if (lattice != LBM_D3Q19 && lattice != LBM_D3Q27) return LBM_ERR_UNSUPPORTED;
    if (lattice == LBM_D3Q27 &&
        (physics != LBM_PHYS_FLUID || (precision != LBM_FP32 && precision != LBM_FP64) ||
         grid->wall_model != LBM_WALL_BOUNCE_BACK || (forcing && forcing->rho_ref != 0.0)))
        return LBM_ERR_UNSUPPORTED;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || grid->ny > 65535 || grid->nz > 65535) return LBM_ERR_ARG;
    const double cells = (double)grid->nx * grid->ny * grid->nz;
    if (cells >= 2147483648.0) return LBM_ERR_ARG;
    if (!(relax->omega > 0.0 && relax->omega < 2.0)) return LBM_ERR_ARG;
    if (relax->omega_bulk != 1.0 || relax->omega_3 != 1.0 || relax->omega_4 != 1.0) return LBM_ERR_UNSUPPORTED;
    if ((int)physics < 0 || (int)physics > 3) return LBM_ERR_ARG;
    if ((int)precision < 0 || (int)precision > 3) return LBM_ERR_ARG;
    if (physics != LBM_PHYS_FLUID && (precision == LBM_FP16_SHIFTED || precision == LBM_BF16_SHIFTED))
        return LBM_ERR_UNSUPPORTED;
    if (physics != LBM_PHYS_FLUID && !phys) return LBM_ERR_ARG;
    if (physics == LBM_PHYS_MHD && !(phys->tau_m > 0.5)) return LBM_ERR_ARG;
    if (physics == LBM_PHYS_CGM) {
        if (!(phys->alpha_r >= 0.0 && phys->alpha_r < 1.0 && phys->alpha_b >= 0.0 && phys->alpha_b < 1.0))
            return LBM_ERR_ARG;
        const bool lid = (grid->periodic_mask & 2u) == 0 &&
                         (grid->lid_u[0] != 0.0 || grid->lid_u[1] != 0.0 || grid->lid_u[2] != 0.0);
        if (lid) return LBM_ERR_UNSUPPORTED;
    }
    if (physics == LBM_PHYS_SC && !std::isfinite(phys->G)) return LBM_ERR_ARG;
    if (grid->wall_model != LBM_WALL_BOUNCE_BACK && grid->wall_model != LBM_WALL_REGULARIZED) return LBM_ERR_ARG;
    if (relax->moment_space != LBM_MOMENTS_CENTRAL && relax->moment_space != LBM_MOMENTS_RAW) return LBM_ERR_ARG;
    if (relax->moment_space == LBM_MOMENTS_RAW &&
        (physics != LBM_PHYS_FLUID || grid->wall_model != LBM_WALL_BOUNCE_BACK))
        return LBM_ERR_UNSUPPORTED;
    if (grid->wall_model == LBM_WALL_REGULARIZED &&
        (physics != LBM_PHYS_FLUID || (grid->periodic_mask & 7u) != 5u || grid->ny < 3))
        return LBM_ERR_UNSUPPORTED;
    if (forcing && forcing->rho_ref != 0.0 && physics != LBM_PHYS_CGM && physics != LBM_PHYS_SC)
        return LBM_ERR_UNSUPPORTED;
    if (physics == LBM_PHYS_MHD) {
        const bool lid = (grid->periodic_mask & 2u) == 0 &&
                         (grid->lid_u[0] != 0.0 || grid->lid_u[1] != 0.0 || grid->lid_u[2] != 0.0);
        if (lid) return LBM_ERR_UNSUPPORTED;
    }

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_OOM;
    c->grid = *grid;
    c->relax = *relax;
    if (forcing)
        c->forcing = *forcing;
    else
        std::memset(&c->forcing, 0, sizeof(c->forcing));
    c->physics = physics;
    if (phys)
        c->phys = *phys;
    else
        std::memset(&c->phys, 0, sizeof(c->phys));
    c->prec = precision;
    c->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);
    c->box.nx = grid->nx;
    c->box.ny = grid->ny;
    c->box.nz = grid->nz;
    c->box.periodic = grid->periodic_mask & 7u;
    c->box.n = (size_t)grid->nx * grid->ny * grid->nz;
    c->elem = precision == LBM_FP64 ? 8 : (precision == LBM_FP32 ? 4 : 2);
    c->q = lattice == LBM_D3Q27 ? 27 : 19;
    c->planes = c->q == 27 ? 27
                           : ((physics == LBM_PHYS_FLUID || physics == LBM_PHYS_SC) ? 19 : (physics == LBM_PHYS_MHD ? 40 : 24));
    c->alloc = g_alloc;
    c->release = g_release;
    c->user = g_user;
    c->block_x = grid->nx >= 256 ? 256 : (grid->nx >= 128 ? 128 : (grid->nx >= 64 ? 64 : 32));

    const size_t state = (size_t)c->planes * c->box.n * c->elem;
    const size_t cb = compute_bytes(c);
    const size_t plane = (size_t)grid->nx * grid->ny;
    size_t kz = SLAB_TARGET_CELLS / plane;
    if (kz < 1) kz = 1;
    if (kz > (size_t)grid->nz) kz = (size_t)grid->nz;
    const int nzs = (int)kz;
    c->staging_cells = plane * kz;
    c->buf[0] = dev_alloc(c, state);
    c->buf[1] = dev_alloc(c, state);
    c->uprev = dev_alloc(c, 3 * c->box.n * cb);
    c->partials = (double*)dev_alloc(c, sizeof(double) * lbm::RED_WIDTH * lbm::RED_BLOCKS);
    c->result = (double*)dev_alloc(c, sizeof(double) * lbm::RED_WIDTH);
    c->staging = (double*)dev_alloc(c, sizeof(double) * 2 * 8 * c->staging_cells);
    const bool has_phi = physics == LBM_PHYS_CGM || physics == LBM_PHYS_SC;
    // scratch: psi (Shan-Chen); phi and the red density (colour gradient)
    if (has_phi) c->phi = dev_alloc(c, (physics == LBM_PHYS_CGM ? 2 : 1) * c->box.n * cb);
    c->status = (int*)dev_alloc(c, 256);
    bool ok = c->buf[0] && c->buf[1] && c->uprev && c->partials && c->result && c->staging && c->status &&
              (!has_phi || c->phi) && make_copy_stream(c);
    if (ok && cudaMallocHost((void**)&c->result_host, sizeof(double) * lbm::RED_WIDTH) != cudaSuccess) {
        cudaGetLastError();
        c->result_host = nullptr;
        ok = false;
    }
    if (!ok) {
        release_all(c);
        delete c;
        return LBM_ERR_OOM;
    }
    // Launch shape default: direct pulls, one node per thread (lbm_autotune
    // or lbm_set_launch_shape may select the staged or paired kernels).
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    c->tma_stages = lbm::fluid_tma_max_stages(c, 1);
    c->variant = 0;
    // Rest state (rho = 1, u = 0; CGM: blue fluid of unit density).
    cudaError_t e = cudaMemsetAsync(c->status, 0, 256, c->stream);
    for (int z0 = 0; z0 < grid->nz && e == cudaSuccess; z0 += nzs) {
        const int k = (z0 + nzs <= grid->nz) ? nzs : grid->nz - z0;
        e = phys_init(c, c->staging, z0, k, true);
    }

    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cuda_fail(c, e, "lbm_create");
        release_all(c);
        delete c;
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c || !c->owns) return;  // views of a batch are owned by the batch
    cudaStreamSynchronize(c->stream);
    if (c->batch) {
        lbm_internal_free_batch_tables(c);
        lbm::batch_destroy(c);
    }
    release_all(c);
    delete c;
}

lbm_status lbm_init_fields(lbm_ctx* c, const double* rho, const double* u, const double* phase, const double* B) {
    if (!c || !rho) return LBM_ERR_ARG;
    if (c->batch) return fail(c, LBM_ERR_ARG, "use the per-domain view of a batch (lbm_batch_domain)%s");
    if (c->physics == LBM_PHYS_CGM && !phase) return fail(c, LBM_ERR_ARG, "CGM needs the phase field%s");
    const size_t n = c->box.n, plane = (size_t)c->box.nx * c->box.ny;
    const int nzs = slab_planes(c);
    // Two slabs in turn: the copies of slab j (copy stream) overlap the
    // initialisation kernel of slab j - 1 (the context's stream).
    cudaStream_t cs = c->copy_stream;
    cudaError_t e = cudaEventRecord(c->fields_start, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, c->fields_start, 0);
    for (int z0 = 0, j = 0; z0 < c->box.nz && e == cudaSuccess; z0 += nzs, ++j) {
        const int k = (z0 + nzs <= c->box.nz) ? nzs : c->box.nz - z0;
        const size_t m = plane * k, off = plane * z0;
        const int b = j & 1;
        double* s = slab_buf(c, b);
        if (j >= 2) e = cudaStreamWaitEvent(cs, c->slab_free[b], 0);  // slab j - 2's kernel has read it
        if (e == cudaSuccess) e = cudaMemcpyAsync(s, rho + off, m * 8, cudaMemcpyDefault, cs);
        for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
            if (u)
                e = cudaMemcpyAsync(s + (1 + a) * m, u + a * n + off, m * 8, cudaMemcpyDefault, cs);
            else
                e = cudaMemsetAsync(s + (1 + a) * m, 0, m * 8, cs);
        }
        if (e == cudaSuccess && c->physics == LBM_PHYS_CGM)
            e = cudaMemcpyAsync(s + 4 * m, phase + off, m * 8, cudaMemcpyDefault, cs);
        for (int a = 0; a < 3 && e == cudaSuccess && c->physics == LBM_PHYS_MHD; ++a) {
            if (B)
                e = cudaMemcpyAsync(s + (5 + a) * m, B + a * n + off, m * 8, cudaMemcpyDefault, cs);
            else
                e = cudaMemsetAsync(s + (5 + a) * m, 0, m * 8, cs);
        }
        if (e == cudaSuccess) e = cudaEventRecord(c->slab_ready[b], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->slab_ready[b], 0);
        if (e == cudaSuccess) e = phys_init(c, s, z0, k, false);
        if (e == cudaSuccess) e = cudaEventRecord(c->slab_free[b], c->stream);
    }
    if (e != cudaSuccess) {
        cudaStreamSynchronize(cs);
        cudaStreamSynchronize(c->stream);
        return cuda_fail(c, e, "lbm_init_fields");
    }
    c->have_prev = false;
    e = cudaStreamSynchronize(c->stream);  // it waited for every slab's copies
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_init_fields");
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, long n) {
    if (!c || n < 0) return LBM_ERR_ARG;
    if (c->batch) return lbm_batch_step(c, n);
    if (!c->owns) return fail(c, LBM_ERR_UNSUPPORTED, "a batch view steps with its batch (lbm_batch_step)%s");
    if (n == 0) return LBM_OK;
    cudaError_t e = phys_step(c, n);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step");
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_sync");
    const lbm_status st = device_status(c);
    if (st != LBM_OK) return st;
    return lbm_internal_batch_status(c);
}

lbm_status lbm_fields(lbm_ctx* c, double* rho, double* u, double* phase, double* B) {
    if (!c) return LBM_ERR_ARG;
    if (c->batch) return fail(c, LBM_ERR_ARG, "use the per-domain view of a batch (lbm_batch_domain)%s");
    const size_t n = c->box.n, plane = (size_t)c->box.nx * c->box.ny;
    const int nzs = slab_planes(c);
    // Two slabs in turn: the field kernel of slab j (the context's stream)
    // overlaps the copies of slab j - 1 (copy stream).
    cudaStream_t cs = c->copy_stream;
    cudaError_t e = cudaSuccess;
    for (int z0 = 0, j = 0; z0 < c->box.nz && e == cudaSuccess; z0 += nzs, ++j) {
        const int k = (z0 + nzs <= c->box.nz) ? nzs : c->box.nz - z0;
        const size_t m = plane * k, off = plane * z0;
        const int b = j & 1;
        double* s = slab_buf(c, b);
        if (j >= 2) e = cudaStreamWaitEvent(c->stream, c->slab_free[b], 0);  // slab j - 2 copied out
        if (e == cudaSuccess) e = phys_fields(c, s, z0, k);
        if (e == cudaSuccess) e = cudaEventRecord(c->slab_ready[b], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, c->slab_ready[b], 0);
        if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho + off, s, m * 8, cudaMemcpyDefault, cs);
        for (int a = 0; a < 3 && e == cudaSuccess && u; ++a)
            e = cudaMemcpyAsync(u + a * n + off, s + (1 + a) * m, m * 8, cudaMemcpyDefault, cs);
        if (e == cudaSuccess && phase && (c->physics == LBM_PHYS_CGM || c->physics == LBM_PHYS_SC))
            e = cudaMemcpyAsync(phase + off, s + 4 * m, m * 8, cudaMemcpyDefault, cs);
        for (int a = 0; a < 3 && e == cudaSuccess && B && c->physics == LBM_PHYS_MHD; ++a)
            e = cudaMemcpyAsync(B + a * n + off, s + (5 + a) * m, m * 8, cudaMemcpyDefault, cs);
        if (e == cudaSuccess) e = cudaEventRecord(c->slab_free[b], cs);
    }
    // the caller's buffers are complete once the copy stream has drained
    const cudaError_t e1 = cudaStreamSynchronize(cs);
    const cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_fields");
    return device_status(c);
}

lbm_status lbm_reduce(lbm_ctx* c, double* out_mass, double* out_mom, double* out_residual) {
    if (!c) return LBM_ERR_ARG;
    if (c->batch) return fail(c, LBM_ERR_ARG, "use the per-domain view of a batch (lbm_batch_domain)%s");
    cudaError_t e = phys_reduce(c, true);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->result_host, c->result, sizeof(double) * lbm::RED_WIDTH, cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_reduce");
    const lbm_status dst = device_status(c);
    if (dst != LBM_OK) return dst;
    const double* r = c->result_host;
    const bool had_prev = c->have_prev;
    c->have_prev = true;
    if (out_mass) *out_mass = r[0];
    if (out_mom) {
        out_mom[0] = r[1];
        out_mom[1] = r[2];
        out_mom[2] = r[3];
    }
    if (out_residual) *out_residual = had_prev ? (r[5] > 0 ? std::sqrt(r[4] / r[5]) : (r[4] > 0 ? INFINITY : 0.0)) : -1.0;
    if (r[6] > 0.0) {
        char buf[128];
        std::snprintf(buf, sizeof(buf), "%.0f nodes with non-finite values or rho <= 0", r[6]);
        c->err = buf;
        c->have_prev = false;
        return LBM_ERR_DIVERGED;
    }
    return LBM_OK;
}

lbm_status lbm_run_to_steady(lbm_ctx* c, long max_steps, long check_every, double tol, long* steps_done,
                             double* residual) {
    if (!c || max_steps < 0 || check_every < 1 || !(tol > 0)) return LBM_ERR_ARG;
    if (c->batch || !c->owns) return fail(c, LBM_ERR_UNSUPPORTED, "steady driver runs on single-domain contexts%s");
    // residual = ||u^n - u^(n-k)|| / (k ||u^n||), k = check_every: the mean
    // per-step rate of change over the check interval
    long done = 0;
    double res = -1.0;
    c->have_prev = false;
    lbm_status s = lbm_reduce(c, nullptr, nullptr, nullptr);  // records u at the start
    while (s == LBM_OK && done < max_steps) {
        long k = check_every;
        if (done + k > max_steps) k = max_steps - done;
        s = lbm_step(c, k);
        if (s != LBM_OK) break;
        done += k;
        double r = -1.0;
        s = lbm_reduce(c, nullptr, nullptr, &r);  // compares with the previous check, records u
        if (s != LBM_OK) break;
        res = r / (double)k;
        if (res <= tol) break;
    }
    if (steps_done) *steps_done = done;
    if (residual) *residual = res;
    return s;
}

size_t lbm_state_bytes(const lbm_ctx* c) {
    if (!c) return 0;
    if (c->batch) return lbm_internal_batch_state_elems(c) * c->elem;
    return (size_t)c->planes * c->box.n * c->elem;
}

lbm_status lbm_get_populations(lbm_ctx* c, void* dst, size_t bytes) {
    if (!c || !dst || bytes != lbm_state_bytes(c)) return LBM_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(dst, c->buf[c->cur], bytes, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_get_populations");
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* c, const void* src, size_t bytes) {
    if (!c || !src || bytes != lbm_state_bytes(c)) return LBM_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(c->buf[c->cur], src, bytes, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_set_populations");
    c->have_prev = false;
    return LBM_OK;
}

}  // extern "C"
