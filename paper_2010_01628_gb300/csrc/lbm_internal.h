// lbm_internal.h -- host-side declarations shared by the library's .cu files.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

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
    int planes;       // stored planes per state copy (19 fluid, 40 MHD, 38 CGM)
    void* buf[2];     // state copies (pull A-B); buf[cur] is current
    int cur;
    void* phi;        // CGM order parameter (compute type)
    void* uprev;      // velocity recorded by the last reduction (compute type, 3 planes)
    bool have_prev;
    double* partials; // per-block reduction partials
    int npartials;
    double* result;   // reduction result (device)
    double* result_host;
    double* staging;  // FP64 field slab
    size_t staging_cells;
    lbm_alloc_fn alloc;
    lbm_free_fn release;
    void* user;
    int block_x;      // threads per block along x for the step kernels
    std::string err;
};

namespace lbm {

// Number of doubles per reduction partial.
constexpr int RED_WIDTH = 8;  // mass, mom x/y/z, |du|^2, |u|^2, bad-node count, spare
constexpr int RED_BLOCKS = 1216;  // 152 SMs x 8
constexpr int RED_THREADS = 256;

// Kernel launchers, one per physics module; each returns cudaGetLastError().
cudaError_t fluid_step(lbm_ctx* c, long n);
cudaError_t fluid_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform);
cudaError_t fluid_fields(lbm_ctx* c, double* slab, int z0, int nzs);
cudaError_t fluid_reduce(lbm_ctx* c, bool record);

cudaError_t mhd_step(lbm_ctx* c, long n);
cudaError_t mhd_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform);
cudaError_t mhd_fields(lbm_ctx* c, double* slab, int z0, int nzs);
cudaError_t mhd_reduce(lbm_ctx* c, bool record);

cudaError_t cgm_step(lbm_ctx* c, long n);
cudaError_t cgm_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform);
cudaError_t cgm_fields(lbm_ctx* c, double* slab, int z0, int nzs);
cudaError_t cgm_reduce(lbm_ctx* c, bool record);

// Sum RED_BLOCKS partials into c->result (deterministic order).
cudaError_t reduce_finalize(lbm_ctx* c);

inline dim3 step_grid(const Box& b, int bx) { return dim3((unsigned)((b.nx + bx - 1) / bx), (unsigned)b.ny, (unsigned)b.nz); }

}  // namespace lbm
