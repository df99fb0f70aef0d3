// lbm_internal.h -- host-side declarations shared by the library's .cu files.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

struct BatchState;

struct lbm_ctx {
    lbm_grid grid;
    lbm_relax relax;
    lbm_forcing forcing;
    lbm_physics physics;
    lbm_physparams phys;
    lbm_precision prec;
    cudaStream_t stream;
    int device;
    lbm::Box box;
    size_t elem;      // bytes per stored population value
    int planes;       // stored planes per state copy (19 fluid and Shan-Chen, 27 D3Q27, 40 MHD, 38 CGM)
    int q = 19;       // lattice: 19 or 27
    void* buf[2];     // state copies (pull A-B); buf[cur] is current
    int cur;
    void* phi;        // CGM order parameter / Shan-Chen pseudopotential (compute type)
    void* uprev;      // velocity recorded by the last reduction (compute type, 3 planes)
    bool have_prev;
    double* partials; // per-block reduction partials
    int npartials;
    double* result;   // reduction result (device)
    double* result_host;
    double* staging;  // two FP64 field slabs of 8 planes x staging_cells, back to back
    size_t staging_cells;
    cudaStream_t copy_stream = nullptr;  // host<->device field copies, overlapping the slab kernels
    cudaEvent_t slab_ready[2] = {nullptr, nullptr};  // a slab's copies (upload) or kernel (download) done
    cudaEvent_t slab_free[2] = {nullptr, nullptr};   // a slab's kernel (upload) or copies (download) done
    cudaEvent_t fields_start = nullptr;              // orders the copy stream after earlier work
    lbm_alloc_fn alloc;
    lbm_free_fn release;
    void* user;
    int block_x;      // threads per block along x for the step kernels
    int variant = 0;  // 0 direct pulls, 1 TMA-staged rows, 2 16-bit x-pairs, 3 fused Shan-Chen, 4 16-bit z-pairs
    int tma_stages = 0;
    int tma_ctas = 1; // CTAs per SM of the TMA-staged kernel
    int zchunk = 32;  // planes per CTA of the fused Shan-Chen kernel (variant 3)
    int fused_threads = 256;  // threads per CTA of that kernel (32 x 8 or 32 x 16)
    int sms = 0;
    int* status = nullptr;  // device status word written by bounded waits
    std::string err;
    bool owns = true;            // false for the per-domain views of a batch
    lbm_ctx* parent = nullptr;   // the batch a view belongs to
    BatchState* batch = nullptr; // set on a batch context
};

// Helpers shared between the C-ABI translation units.
void* lbm_internal_dev_alloc(lbm_ctx* c, size_t bytes);
void lbm_internal_get_allocator(lbm_alloc_fn* a, lbm_free_fn* r, void** user);
void lbm_internal_dev_free(lbm_ctx* c, void* p);
lbm_status lbm_internal_alloc_batch(lbm_ctx* c, size_t state_elems, size_t cells, size_t max_plane);
void lbm_internal_release(lbm_ctx* c);
cudaError_t lbm_internal_init_slab(lbm_ctx* c, int z0, int nzs, bool uniform);
cudaError_t lbm_internal_step(lbm_ctx* c, long n, bool dry);
lbm_status lbm_internal_batch_status(lbm_ctx* c);
lbm_status lbm_internal_alloc_batch_tables(lbm_ctx* c);
size_t lbm_internal_batch_state_elems(const lbm_ctx* c);
void lbm_internal_free_batch_tables(lbm_ctx* c);

namespace lbm {

// Number of doubles per reduction partial.
constexpr int RED_WIDTH = 8;  // mass, mom x/y/z, |du|^2, |u|^2, bad-node count, spare
constexpr int RED_BLOCKS = 1216;  // 152 SMs x 8
constexpr int RED_THREADS = 256;

// Kernel launchers, one per physics module; each returns cudaGetLastError().
// A "dry" step reads the current state and writes the other buffer without
// making it current (timing runs of the autotuner leave the state unchanged).
cudaError_t fluid_step(lbm_ctx* c, long n, bool dry = false);
// Largest stage count of the TMA-staged kernel that fits `ctas` CTAs per SM (0
// if the geometry does not allow the variant).
int fluid_tma_max_stages(const lbm_ctx* c, int ctas);
// The 16-bit single-phase step with two nodes per thread and packed FP32x2
// arithmetic (launch variants 2 and 4): D3Q19 central moments, bounce-back walls.
// Threads per CTA of the z-pair kernel (launch variant 4), fixed by its launch bounds.
constexpr int ZPAIR_MAX_THREADS = 128;
inline bool packed16_ok(const lbm_ctx* c) {
    return c->physics == LBM_PHYS_FLUID && (c->prec == LBM_FP16_SHIFTED || c->prec == LBM_BF16_SHIFTED) &&
           c->grid.wall_model == LBM_WALL_BOUNCE_BACK && c->relax.moment_space == LBM_MOMENTS_CENTRAL && c->q == 19;
}
cudaError_t fluid_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform);
cudaError_t fluid_fields(lbm_ctx* c, double* slab, int z0, int nzs);
cudaError_t fluid_reduce(lbm_ctx* c, bool record);

cudaError_t mhd_step(lbm_ctx* c, long n, bool dry = false);
cudaError_t mhd_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform);
cudaError_t mhd_fields(lbm_ctx* c, double* slab, int z0, int nzs);
cudaError_t mhd_reduce(lbm_ctx* c, bool record);

cudaError_t cgm_step(lbm_ctx* c, long n, bool dry = false);
cudaError_t cgm_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform);
cudaError_t cgm_fields(lbm_ctx* c, double* slab, int z0, int nzs);
cudaError_t cgm_reduce(lbm_ctx* c, bool record);

// D3Q27 single phase (lbm_q27.cu).
cudaError_t q27_step(lbm_ctx* c, long n, bool dry = false);
cudaError_t q27_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform);
cudaError_t q27_fields(lbm_ctx* c, double* slab, int z0, int nzs);
cudaError_t q27_reduce(lbm_ctx* c, bool record);

// Shan-Chen (lbm_sc.cu); initialisation is the single-phase one.
cudaError_t sc_step(lbm_ctx* c, long n, bool dry = false);
cudaError_t sc_fields(lbm_ctx* c, double* slab, int z0, int nzs);
cudaError_t sc_reduce(lbm_ctx* c, bool record);

// Sum RED_BLOCKS partials into c->result (deterministic order).
cudaError_t reduce_finalize(lbm_ctx* c);

// Batched persistent kernel (lbm_batch.cu).
cudaError_t batch_time_config(lbm_ctx* c, int threads, int ctas_per_sm, long steps, float* ms);
cudaError_t batch_apply_config(lbm_ctx* c, int threads, int ctas_per_sm);
void batch_destroy(lbm_ctx* c);

inline dim3 step_grid(const Box& b, int bx) { return dim3((unsigned)((b.nx + bx - 1) / bx), (unsigned)b.ny, (unsigned)b.nz); }

}  // namespace lbm
