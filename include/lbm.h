/*
 * lbm.h -- C ABI of the GB300 (sm_103a) D3Q19 central-moment lattice Boltzmann
 * library (liblbm.so).
 *
 * Method: De Rosis & Coreixas, "Multiphysics flow simulations using D3Q19
 * lattice Boltzmann methods based on central moments", arXiv:2010.01628.
 * One time step streams the 19 populations (Eq. streaming), takes rho and u
 * (Eq. macro, with +F/2 when a force acts, App. E), relaxes the central
 * moments toward the Galilean-invariant equilibrium with the forcing terms
 * (Eq. eq:posColl0 and the list after it), and rebuilds the populations by the
 * two-step transform of App. C (Eqs. rawQ19, pdfQ19).  Physics modules add the
 * Lorentz force with magnetic populations (Sec. III.F) or the colour-gradient
 * two-phase operator (App. E).
 *
 * Conventions shared by every entry point:
 *  - Lattice units (dx = dt = 1), c_s^2 = 1/3, omega = 1/(nu/c_s^2 + 1/2).
 *  - Fields are FP64, layout [nz][ny][nx] with x fastest; vectors (u, B) are
 *    three such planes back to back (x, y, z components).
 *  - Field pointers may be host memory (pageable or pinned) or device memory
 *    of the context's GPU; the library copies with cudaMemcpyAsync on the
 *    context stream and synchronises before returning.
 *  - The caller owns every pointer it passes in.  The library owns its device
 *    buffers (populations, scratch), obtained from the allocator installed with
 *    lbm_set_allocator, else cudaMalloc.
 *  - Every call returns an lbm_status; nothing aborts or traps, and nothing
 *    throws across the ABI.  lbm_last_error() gives a one-line reason.
 *  - Kernels run asynchronously on the context stream.  lbm_step() returns
 *    after enqueueing; errors of earlier launches surface at the next call
 *    that synchronises (fields, reduce, sync, populations).
 *  - Time-step order: the stored state is the post-collision populations; a
 *    step gathers them (stream + boundaries) and collides.  The initial state
 *    is the equilibrium of the given fields.  Reported fields are the moments
 *    of the gathered (post-stream) populations.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,         /* invalid argument (sizes, rates, null pointers) */
    LBM_ERR_OOM = 2,         /* device allocation failed */
    LBM_ERR_CUDA = 3,        /* a CUDA call failed */
    LBM_ERR_DIVERGED = 4,    /* NaN/Inf or rho <= 0 found by a reduction */
    LBM_ERR_TIMEOUT = 5,     /* a bounded device wait (batch grid barrier) ran out */
    LBM_ERR_UNSUPPORTED = 6  /* valid request this build does not implement */
} lbm_status;

/* Velocity sets.  LBM_D3Q19: the paper's lattice (Sec. II.A).  LBM_D3Q27: the
 * App. D lattice (single phase, FP64 or FP32, half-way bounce-back walls,
 * central or raw moments, direct launch shape), used for the App. D cost
 * comparison. */
typedef enum { LBM_D3Q19 = 0, LBM_D3Q27 = 1 } lbm_lattice;

/* Population storage.  FP64 and FP32 store f_i - w_i (shifted by the rest
 * equilibrium of rho0 = 1) and compute in their own type.  The 16-bit formats
 * store (f_i - w_i)/w_i and compute in FP32 registers. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16_SHIFTED = 2, LBM_BF16_SHIFTED = 3 } lbm_precision;

typedef enum {
    LBM_PHYS_FLUID = 0, /* single phase, body force F = rho g (Sec. II)           */
    LBM_PHYS_MHD = 1,   /* + D3Q7 magnetic populations, F = j x b (Sec. III.F)    */
    LBM_PHYS_CGM = 2,   /* colour-gradient two-phase (App. E)                     */
    LBM_PHYS_SC = 3     /* Shan-Chen pseudopotential multiphase (Sec. III.G)      */
} lbm_physics;

/* Wall models.  LBM_WALL_BOUNCE_BACK: half-way bounce-back, the wall midway
 * between the boundary node and the next (virtual) node.  LBM_WALL_REGULARIZED:
 * the regularized on-node walls the paper imposes (Sec. III opening paragraph,
 * citing Latt, Chopard, Malaspinas, Deville and Michler, Phys. Rev. E 77,
 * 056703 (2008)): the wall lies on the boundary nodes y = 0 and y = ny - 1,
 * whose populations are rebuilt from rho (from the known populations), the wall
 * velocity and the non-equilibrium stress; straight channel walls only
 * (LBM_PHYS_FLUID, walls on y, x and z periodic, ny >= 3). */
typedef enum { LBM_WALL_BOUNCE_BACK = 0, LBM_WALL_REGULARIZED = 1 } lbm_wall_model;

/* Box geometry.  A periodic axis wraps; a non-periodic axis has no-slip walls
 * at both ends, of the given wall model.  lid_u is the velocity of the +y wall
 * (bounce-back: Ladd's moving-wall term with rho_w = 1; regularized: the
 * velocity of the y = ny - 1 nodes); it is ignored if y is periodic. */
typedef struct {
    int nx, ny, nz;
    unsigned periodic_mask; /* bit 0: x, bit 1: y, bit 2: z */
    double lid_u[3];
    int wall_model;         /* lbm_wall_model */
} lbm_grid;

/* Moment space of the collision.  LBM_MOMENTS_CENTRAL: the paper's central
 * moments (Sec. II.B).  LBM_MOMENTS_RAW: the raw-moment variant of App. C
 * (N = I, the printed post-collision list; its forcing enters at first and
 * third order only), single phase with half-way bounce-back walls, direct
 * launch shape only. */
typedef enum { LBM_MOMENTS_CENTRAL = 0, LBM_MOMENTS_RAW = 1 } lbm_moment_space;

/* Diagonal relaxation matrix K of Sec. II.B: omega on the five deviatoric
 * second-order CMs; omega_bulk on the trace (k4); omega_3 on k10..k15;
 * omega_4 on k16..k18.  The paper sets omega_bulk = omega_3 = omega_4 = 1,
 * the only values this build accepts (others give LBM_ERR_UNSUPPORTED). */
typedef struct {
    double omega, omega_bulk, omega_3, omega_4;
    int moment_space; /* lbm_moment_space */
} lbm_relax;

/* Body force F = (rho - rho_ref) g (Eq. eq:posColl0): a constant acceleration
 * for rho_ref = 0; the Rayleigh-Taylor test of Sec. III.H drives its two fluids
 * with rho_ref = (rho_h + rho_l)/2.  rho_ref != 0 is accepted by the two-phase
 * modules (LBM_PHYS_CGM, LBM_PHYS_SC, and colour-gradient batches); the other
 * modules return LBM_ERR_UNSUPPORTED for it. */
typedef struct {
    double g[3];
    double rho_ref;
} lbm_forcing;

/* Physics-module parameters.
 * MHD (Sec. III.F): tau_m is the relaxation time of the D3Q7 magnetic
 *   populations (eta = (tau_m - 1/2)/4); b_wall is the field imposed at the
 *   walls (anti-bounce-back).
 * CGM (App. E): alpha_r, alpha_b set phi_i(alpha) and the density ratio
 *   rho_r0/rho_b0 = (1 - alpha_b)/(1 - alpha_r); A is the perturbation
 *   amplitude (sigma = (4/9) A / omega); beta the recolouring parameter.
 * Shan-Chen (Sec. III.G): G is the interaction strength of the force
 *   F = -G psi(x) sum_i w_i c_i psi(x + c_i), psi = 1 - exp(-rho) (the static
 *   bubble uses G = -5); a neighbour behind a wall contributes the node's own
 *   psi. */
typedef struct {
    double tau_m;
    double b_wall[3];
    double alpha_r, alpha_b, A, beta;
    double G;
} lbm_physparams;

/* Device-memory provider.  alloc returns a device pointer of at least `bytes`
 * (256-byte aligned) usable on `stream`, or NULL; free releases it.  Passing
 * NULL for both restores cudaMalloc/cudaFree.  Applies to contexts created
 * afterwards; a context frees with the provider it allocated with. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*lbm_free_fn)(void *ptr, void *stream, void *user);
lbm_status lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void *user);

/* Create a solver on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream); all work of the context is
 * ordered on it.  grid sizes >= 1 with nx*ny*nz < 2^31; 0 < omega < 2.
 * Populations start at rest (rho = 1, u = 0) until lbm_init_fields. */
lbm_status lbm_create(lbm_ctx **out, const lbm_grid *grid, lbm_lattice lattice, const lbm_relax *relax,
                      const lbm_forcing *forcing, lbm_physics physics, const lbm_physparams *phys,
                      lbm_precision precision, void *cuda_stream);

/* Set the populations to the equilibrium of the given fields (Sec. III
 * opening paragraph: Eq. eq:EqQ19RM; App. E's h_eq for CGM; the magnetic
 * equilibrium for MHD).  rho: [n]; u: [3n] or NULL (= 0); phase: [n], CGM
 * only, the order parameter phi of Eq. eq:order; B: [3n], MHD only. */
lbm_status lbm_init_fields(lbm_ctx *ctx, const double *rho, const double *u, const double *phase, const double *B);

/* Enqueue n time steps on the context stream (n >= 0). */
lbm_status lbm_step(lbm_ctx *ctx, long n);

/* Macroscopic fields of the current state (any pointer may be NULL = skip):
 * rho [n]; u [3n] (with +F/2); phase [n] (CGM: the order parameter; Shan-Chen:
 * the pseudopotential psi); B [3n] (MHD).  Synchronises. */
lbm_status lbm_fields(lbm_ctx *ctx, double *rho, double *u, double *phase, double *B);

/* FP64 reductions over all nodes of the current state: total mass sum rho,
 * total momentum sum rho u, and the residual ||u - u_prev||_2 / ||u||_2
 * against the velocity recorded by the previous lbm_reduce call on this
 * context (-1 on the first call).  Records u for the next call.  Returns
 * LBM_ERR_DIVERGED if any node has a non-finite value or rho <= 0.  Any output
 * pointer may be NULL.  Synchronises. */
lbm_status lbm_reduce(lbm_ctx *ctx, double *out_mass, double *out_mom, double *out_residual);

/* Steady-state driver: steps until the residual ||u^n - u^(n-k)||_2 /
 * (k ||u^n||_2) over the check interval k = check_every (the mean per-step
 * relative change, FP64 sums over all nodes) is <= tol, or until max_steps.
 * Reports the steps taken and the last residual. */
lbm_status lbm_run_to_steady(lbm_ctx *ctx, long max_steps, long check_every, double tol, long *steps_done,
                             double *residual);

/* Wait for all enqueued work; reports errors of earlier launches. */
lbm_status lbm_sync(lbm_ctx *ctx);

/* Raw population storage (checkpoint/restart).  Size in bytes of one copy of
 * the state; the layout is the storage format (structure of arrays, planes of
 * n values in direction order, the stored quantity as documented for
 * lbm_precision; MHD appends 21 magnetic planes.  CGM stores 24 unshifted
 * planes: the 19 total populations f_i, then per node the red fraction
 * a = rho_r / rho, the recolouring vector V (3 planes) and the red rest
 * population; the red population of moving direction i is a f_i + kappa_i c_i.V
 * with kappa = 1/12 (axes) or 1/(24 sqrt 2) (diagonals), blue the rest).
 * dst/src may be host or device pointers. */
size_t lbm_state_bytes(const lbm_ctx *ctx);
lbm_status lbm_get_populations(lbm_ctx *ctx, void *dst, size_t bytes);
lbm_status lbm_set_populations(lbm_ctx *ctx, const void *src, size_t bytes);

/* ---- Batched parameter sweeps ---------------------------------------------
 * Many independent domains (uneven sizes, per-domain omega, force, wall field,
 * density ratio, surface tension) advanced together: each lbm_batch_step runs
 * ONE persistent cooperative kernel that performs all n steps with a
 * bounded-wait grid barrier between steps, replayed from a CUDA graph captured
 * on first use (per step count and buffer parity).  Physics: LBM_PHYS_FLUID,
 * LBM_PHYS_MHD, LBM_PHYS_CGM (App. E colour gradient) or LBM_PHYS_SC (Sec.
 * III.G Shan-Chen); the two-phase steps take two passes per step (order
 * parameter or pseudopotential, then collision) separated by a second grid
 * barrier, and the batch holds their phi and rho_r (psi) planes for all
 * domains; FP64 or FP32.  grids/relax/forcing/phys are arrays of ndomains
 * entries (forcing may be NULL; rho_ref must be 0 except for CGM and SC; phys
 * is required for MHD, CGM and SC, whose tau_m and b_wall, alpha_r, alpha_b,
 * A, beta, or G are taken per domain; the colour gradient and MHD have no
 * moving lid).  Domain d is initialised, read back, reduced and
 * checkpointed through its view (lbm_batch_domain), which accepts
 * lbm_init_fields, lbm_fields, lbm_reduce and lbm_get/set_populations; the view
 * is owned by the batch (lbm_destroy on it does nothing, lbm_step on it is
 * LBM_ERR_UNSUPPORTED).  lbm_step on the batch context equals lbm_batch_step.
 * A barrier wait longer than 2 s ends the kernel; lbm_sync then returns
 * LBM_ERR_TIMEOUT. */
lbm_status lbm_batch_create(lbm_ctx **out, int ndomains, const lbm_grid *grids, const lbm_relax *relax,
                            const lbm_forcing *forcing, lbm_physics physics, const lbm_physparams *phys,
                            lbm_precision precision, void *cuda_stream);
lbm_status lbm_batch_domain(lbm_ctx *batch, int domain, lbm_ctx **view);
lbm_status lbm_batch_step(lbm_ctx *batch, long n);
/* Launch shape of the persistent kernel: threads per CTA, CTAs, whether the
 * launch is replayed from a captured graph, number of tiles per step. */
lbm_status lbm_batch_info(const lbm_ctx *batch, int *threads, int *grid, int *graph, long *tiles);

/* Diagnostic of the bounded device waits: runs a grid barrier that can never
 * complete on the current device with the given limit (0 < timeout_s <= 10)
 * and reports the status word the kernel wrote (LBM_ERR_TIMEOUT expected). */
lbm_status lbm_barrier_selftest(double timeout_s, int *observed);

/* Diagnostic of the bounded mbarrier wait of the TMA-staged kernels (launch
 * variant 1): one thread waits for an mbarrier phase with the given limit
 * (0 < timeout_s <= 10).  arrive = 0: nothing completes the phase and the wait
 * must give up (LBM_ERR_TIMEOUT in *observed); arrive != 0: the thread arrives
 * first and the wait must succeed (LBM_OK).  The device stays usable. */
lbm_status lbm_mbarrier_selftest(double timeout_s, int arrive, int *observed);

/* ---- Autotuner ---------------------------------------------------------------
 * Chooses the launch shape of a context by timed trials that leave its state
 * unchanged: threads per block of the single-domain step kernels, or threads
 * per CTA and CTAs per SM of the batched persistent kernel.  Results are cached
 * in a JSON file (cache_path, may be NULL = no cache) keyed by device, physics,
 * precision and geometry; a cached entry is applied without timing unless
 * force != 0.  Reports the chosen throughput in MLUPS (may be NULL). */
lbm_status lbm_autotune(lbm_ctx *ctx, const char *cache_path, int force, double *mlups);

/* Set the launch shape of a single-domain context by hand (what lbm_autotune
 * chooses): variant 0 = one thread per node pulling straight from global
 * memory (`threads` per block: 32..256, multiple of 32); variant 2 = two
 * x-neighbour nodes per thread with aligned 32-bit accesses (16-bit storage,
 * even nx, single phase); variant 4 = two z-neighbour nodes per thread with
 * plain 2-byte pulls (16-bit storage, single phase); variants 2 and 4 relax
 * both nodes with packed FP32x2 arithmetic (same rounding per node as the
 * scalar FP32 code, different fma contraction); variant 1 = the
 * TMA-staged kernel for single-phase flow (x-rows of 19 planes fetched into
 * shared memory by bulk copies, `stages` rows in flight per CTA, `ctas` CTAs
 * per SM); it needs nx * bytes-per-value to be a multiple of 16 and enough
 * shared memory for 2 stages, else LBM_ERR_UNSUPPORTED; variant 3 = the fused
 * Shan-Chen step (LBM_PHYS_SC only): CTAs of 32 x 8 (`threads` = 256) or
 * 32 x 16 (512, FP32 only) threads march through `stages` z-planes each
 * (0 = 32), keeping the pseudopotential of three planes in shared memory. */
lbm_status lbm_set_launch_shape(lbm_ctx *ctx, int variant, int threads, int stages, int ctas);
lbm_status lbm_get_launch_shape(const lbm_ctx *ctx, int *variant, int *threads, int *stages, int *ctas);

/* ---- Learned warm start ---------------------------------------------------
 * A 3D convolutional network predicts the steady (rho, u) of the lid-driven
 * cavity from the Reynolds number; lbm_cnn_warm_start initialises a solver
 * with the prediction (populations at the equilibrium of the predicted
 * fields) so that it iterates to the steady residual from there instead of
 * from rest.  The network is an addition of this library (the paper has no
 * learned component): 4 layers of 3x3x3 zero-padded convolutions,
 * 16 -> 32 -> 32 -> 32 -> 4 channels, ReLU after the first three, BF16
 * activations and kernel weights on the tensor cores, FP32 master weights,
 * gradients and Adam moments.
 * Inputs per node (16): r = (Re - 550)/450, the node-centre coordinates
 * x, y, z scaled to [-1, 1], 1 on the top (+y, lid) layer of nodes,
 * cos(pi v/2), sin(pi v), cos(pi v) of each coordinate v, r^2, r (y + 1)/2.  Outputs per node:
 * (rho - 1) * 30 and u * 10 (lid speed 0.1 -> 1).
 * Parameters (lbm_cnn_param_count of them): per layer, weights
 * [C_out][C_in][27] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)) then biases [C_out].
 * Fields are FP64 planar ([n] rho, [3n] u), host or device pointers; device
 * pointers of the current device are read in place (each call synchronises
 * before it returns), host ones are copied in first.
 * Errors: LBM_ERR_ARG for null handles or wrong counts, LBM_ERR_OOM, LBM_ERR_CUDA,
 * LBM_ERR_TIMEOUT when a tensor-core pipeline wait ran past its bound (the
 * kernels then drain and free their TMEM; the context stays usable). */
typedef struct lbm_cnn lbm_cnn;
size_t lbm_cnn_param_count(void);
/* init_weights: NULL = deterministic He-uniform initialisation. */
lbm_status lbm_cnn_create(lbm_cnn **out, int nx, int ny, int nz, const float *init_weights, void *cuda_stream);
void lbm_cnn_destroy(lbm_cnn *net);
const char *lbm_cnn_last_error(const lbm_cnn *net);
lbm_status lbm_cnn_set_weights(lbm_cnn *net, const float *w, size_t count);
lbm_status lbm_cnn_get_weights(lbm_cnn *net, float *w, size_t count);
/* Input channels from the Reynolds number (device-side). */
lbm_status lbm_cnn_set_input(lbm_cnn *net, double reynolds);
/* Input channels given explicitly: x [n][16] FP32 (tests). */
lbm_status lbm_cnn_set_input_raw(lbm_cnn *net, const float *x, size_t count);
/* Forward pass; out (optional) receives the [n][4] FP32 outputs. */
lbm_status lbm_cnn_forward(lbm_cnn *net, float *out, size_t count);
/* Loss (mean squared error of the 4 outputs against the scaled fields) and
 * its gradient with respect to all parameters (grad_out optional). */
lbm_status lbm_cnn_gradient(lbm_cnn *net, const double *rho, const double *u, double *loss, float *grad_out,
                            size_t count);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the gradient of the
 * loss against the given steady fields. */
lbm_status lbm_cnn_train_step(lbm_cnn *net, const double *rho, const double *u, float lr, double *loss);
/* Predict for `reynolds` and initialise ctx (same grid) from the prediction. */
lbm_status lbm_cnn_warm_start(lbm_cnn *net, lbm_ctx *ctx, double reynolds);

/* Measured FMA throughput of the current device (independent FMA chains, best
 * of 3): FP64 and FP32 fused multiply-adds per second.  The FP64 step is
 * bound by the FP64 pipe; this is the denominator of its ALU roofline. */
lbm_status lbm_probe_fma_rate(double *fp64_fma_per_s, double *fp32_fma_per_s);

/* Allocation-free FP64 reduction of a single-phase population state that the
 * caller owns (the paper has no counterpart; it exists for callers that may
 * not allocate device memory: applications that own all device memory
 * through their own pool, latency-critical loops where cudaMalloc/cudaFree
 * would stall, code running inside an allocator or memory-pressure callback).
 * populations: device pointer to one state in the storage format of
 *   lbm_get_populations for LBM_PHYS_FLUID with this precision (19 planes).
 * grid, forcing: as for lbm_create (forcing may be NULL = no force;
 *   rho_ref != 0 gives LBM_ERR_UNSUPPORTED).
 * out: device-accessible pointer to 5 doubles, written with the sums over all
 *   nodes of rho, rho u (x, y, z; with +F/2) and the number of nodes with a
 *   non-finite value or rho <= 0, the same quantities lbm_reduce reports.
 * The work is enqueued on cuda_stream; the call does not synchronise.
 * It allocates nothing: its scratch is a fixed 77,824-byte __device__ array
 * (1216 block partials) that every GPU loading the library holds until exit.
 * Grids beyond 2^31 - 1 nodes, or with ny or nz above 65535, are rejected with
 * LBM_ERR_ARG, and so are populations or out that are not device (or managed)
 * memory of the current device (cudaPointerGetAttributes); the sizes of the
 * two buffers cannot be checked here and are the caller's to guarantee.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call before any stream capture.  A cudaDeviceReset, or a context other
 * than the device's primary one, invalidates the kept address: such callers
 * must not use this entry point after the reset or context switch.  All calls
 * share the array: calls that overlap on the GPU race.
 * err/err_len (optional) receive a one-line reason on failure. */
lbm_status lbm_reduce_state_noalloc(const void *populations, lbm_precision precision, const lbm_grid *grid,
                                    const lbm_forcing *forcing, double *out, void *cuda_stream, char *err,
                                    size_t err_len);

void lbm_destroy(lbm_ctx *ctx);
const char *lbm_last_error(const lbm_ctx *ctx);
const char *lbm_status_string(lbm_status s);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
