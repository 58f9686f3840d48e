/*
 * lope.h — C ABI of the GB300 (sm_103a) library for the hot path of
 * locally-oriented programming (LOPe; Rasmussen, Sottile, Nagle, Rasmussen,
 * arXiv:1502.03504): a local function that writes one array element and reads
 * a fixed-width halo around it is applied at every point of a 2D or 3D
 * structured grid, for many time steps.
 *
 * Conventions shared by every call:
 *  - Extents are given slowest axis first; the last axis is contiguous (C
 *    order).  The paper's local offsets U(dx,dy[,dz]) (Sec. 2.2, "LOPe index
 *    notation") map dx to the fastest axis, dy to the next, dz to the slowest.
 *  - Only interior points are stored.  Halo (ghost) values are produced inside
 *    the kernels from the boundary condition; they are never written to memory.
 *  - All field buffers are device memory owned by the caller; handles are owned
 *    by the library.  Pointers must be 16-byte aligned.  Multi-field grids pass
 *    one pointer per field, in the stencil's field order.
 *  - Calls are asynchronous on the given CUDA stream (NULL = legacy default
 *    stream) unless stated otherwise.
 *  - Every call returns a status; on failure lope_last_error() describes it.
 *    There is no CPU fallback: a missing or unusable GPU is an error.
 */
#ifndef LOPE_H
#define LOPE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LOPE_OK = 0,
  LOPE_ERR_INVALID = 1,     /* bad argument (shape, halo, pointer, size)          */
  LOPE_ERR_UNSUPPORTED = 2, /* valid request this build does not implement         */
  LOPE_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed                   */
  LOPE_ERR_ALLOC = 4,       /* host allocation failed / workspace too small        */
  LOPE_ERR_TIMEOUT = 5,     /* a bounded in-kernel wait gave up (device error flag) */
  LOPE_ERR_NUMERIC = 6      /* non-finite result where a finite one was required   */
} lope_status;

typedef enum { LOPE_F64 = 0, LOPE_F32 = 1, LOPE_BF16 = 2 } lope_dtype;

/* Halo contents (Sec. 2.2 "Halo regions": the halo holds boundary-value
 * information).  PERIODIC is the paper's BC=CYCLIC (Sec. 3.2); DIRICHLET holds a
 * fixed value in the halo for every step.  EXTERNAL (slowest axis only) is the
 * halo of one slab of a decomposed grid, the data that HALO_TRANSFER brings
 * from the neighbouring image (Sec. 3.2, Sec. 3.3): the input buffer must hold,
 * right beyond the grid on that side, at least `radius` planes (3D) or rows
 * (2D) of the neighbour's current state -- in[f] - radius * plane .. in[f] is
 * read for the low side, the planes after the grid for the high side.  The
 * caller refreshes them between sweeps (a halo exchange), so such a grid takes
 * nsteps <= 1 per lope_apply; the TMA and direct kernels read it (trapezoid,
 * plane march, batched, adjoint and multi-stage calls return UNSUPPORTED). */
typedef enum { LOPE_BC_PERIODIC = 0, LOPE_BC_DIRICHLET = 1, LOPE_BC_EXTERNAL = 2 } lope_bc;

typedef struct lope_grid lope_grid;
typedef struct lope_stencil lope_stencil;

/* Grid descriptor: a halo-annotated array HALO(lo:*:hi) per axis (Sec. 2.2
 * "Halo regions").  ndim is 2 or 3; extents[ndim] slowest first, each >= 1;
 * halo_lo/halo_hi[ndim] are the declared halo widths (0..4) per axis, which
 * bound the offsets a local function may read (Sec. 3.5: no out-of-bounds
 * indexing).  nfields is 1..3.  All boundaries start PERIODIC.
 * Errors: LOPE_ERR_INVALID for any out-of-range argument or NULL pointer. */
lope_status lope_grid_create(lope_grid** grid, int ndim, const int64_t* extents,
                             const int* halo_lo, const int* halo_hi, lope_dtype storage,
                             int nfields);
void lope_grid_destroy(lope_grid* grid);

/* Boundary condition of one side of one axis (axis 0..ndim-1 slowest first, or
 * -1 for all axes; side 0 low, 1 high, -1 both).  A periodic axis must be
 * periodic on both sides (setting one side of a periodic axis to another kind
 * makes the other side Dirichlet 0).  EXTERNAL is accepted on axis 0 only.
 * Changing the boundary does not change the local function (Sec. 3.4, first
 * advantage).  value is the Dirichlet halo value. */
lope_status lope_set_boundary(lope_grid* grid, int axis, int side, lope_bc kind, double value);

/* Built-in local functions (Sec. 2.2, Fig. 1 and its generalisations):
 *   "jacobi5"   2D, params {c}:      U(0,0) + c (U(-1,0)+U(1,0)+U(0,-1)+U(0,1) - 4 U(0,0));
 *                                    c = 1 is Fig. 1 exactly.
 *   "diff7"     3D, params {c}:      the 7-point analogue, - 6 U(0,0,0).
 *   "star9r2"   2D, params {c}:      U(0,0) + c (L4x + L4y), L4 the fourth-order
 *                                    1D Laplacian (-1/12, 4/3, -5/2, 4/3, -1/12).
 *   "swe_cgrid" 2D, 3 fields (h,u,v), params {dt, g, H}: linearised shallow
 *                                    water on an Arakawa C-grid, forward Euler.
 *   "swe_flux"  2D, 3 fields (eta,u,v), params {dt, g, f, H}: nonlinear shallow
 *                                    water on a C-grid (eta = h - H): flux-form
 *                                    mass, Coriolis on four-face means (corner
 *                                    taps), pressure gradient, centred advection;
 *                                    forward Euler.  A non-linear physics
 *                                    operator with a radius-1 box halo (the
 *                                    kind Sec. 5, Limitations, names).
 * Errors: LOPE_ERR_INVALID for an unknown name or wrong parameter count. */
lope_status lope_stencil_create_builtin(lope_stencil** stencil, const char* name,
                                        const double* params, int nparams);

/* General linear local function U(0,0) = sum_o w[o] U(o) over the box of
 * radius `radius` (1..2): weights has (2r+1)^ndim entries, slowest offset first,
 * i.e. weights[((dz+r)*(2r+1) + dy+r)*(2r+1) + dx+r] (dz only for ndim = 3).
 * Star-shaped tables (all off-axis entries zero) take the TMA kernels; 2D
 * tables with corners take the 2D TMA tiles too, 3D ones the direct kernel. */
lope_status lope_stencil_create_linear(lope_stencil** stencil, int ndim, int radius,
                                       const double* weights);
void lope_stencil_destroy(lope_stencil* stencil);

/* A local function written by the user as source and compiled at run time:
 * the analogue of the paper's compilation of CONCURRENT procedures written in
 * the LOPe index notation (Sec. 2.2; Sec. 4 compiles them source to source),
 * here with NVRTC straight to sm_103a code, into the same kernels the
 * builtins use (TMA tiles / z-march, trapezoid tiles, direct kernel, and the
 * multi-stage schemes).  `body` is the C++ body of the function.  Inside it:
 *   C             the compute type (float for FP32/BF16 storage, double for
 *                 FP64; on the paired TMA path a packed pair of floats);
 *   U(f, dx, dy)  (2D) or U(f, dx, dy, dz) (3D): field f at the local offset,
 *                 dx along the fastest axis (the paper's U(dx,dy)).  The
 *                 declared halo is the contract of Sec. 3.5 (no out-of-bounds
 *                 indexing): a tap whose arguments are integer literals and
 *                 that reads beyond `radius`, reads a field >= nfields, or (box
 *                 = 0) reads a corner makes this call fail with
 *                 LOPE_ERR_INVALID; a computed tap that does so at run time is
 *                 clamped into the halo and lope_sync_status then reports
 *                 LOPE_ERR_INVALID;
 *   P[0..7]       the parameters, in C;
 *   out[f]        must be assigned for every field f < nfields;
 *   add, sub, mul, fma_, C(x), and + - * on C values.
 * Write every product that feeds a sum as fma_() and use add/sub/mul for the
 * rest to get results that are bitwise equal on every kernel path (the
 * compiler may contract packed a*b+c on its own).  box = 0 declares that the
 * function reads only axis-aligned taps (star); box = 1 allows corner taps
 * (2D TMA tiles; 3D box functions take the direct kernel).  The body is
 * compiled on first use per storage type (or by lope_stencil_compile) and runs
 * as trusted code.  Errors: LOPE_ERR_INVALID for out-of-range arguments.  A
 * body that does not compile fails at lope_stencil_compile or at its first
 * launch with LOPE_ERR_INVALID, and lope_last_error() gives the compiler log;
 * without NVRTC (libnvrtc.so.13) those calls return LOPE_ERR_UNSUPPORTED. */
lope_status lope_stencil_create_source(lope_stencil** stencil, int ndim, int radius, int nfields,
                                       int box, const char* body, const double* params,
                                       int nparams);

/* Compile every kernel of a source stencil for one storage type now (NVRTC;
 * no GPU needed), so that no launch compiles and a stream capture does not
 * compile.  A no-op for builtin and linear stencils. */
lope_status lope_stencil_compile(const lope_stencil* stencil, lope_dtype storage);

/* Time-stepping scheme.  A local function is one forward-Euler step E(u) = u +
 * dt F(u) (EULER, the default: a step is one sweep).  RK2 and RK3 are the
 * strong-stability-preserving Runge-Kutta methods of Shu and Osher (1988)
 * written as convex combinations of Euler steps:
 *   RK2: u1 = E(u);  u+ = 1/2 u + 1/2 E(u1)
 *   RK3: u1 = E(u);  u2 = 3/4 u + 1/4 E(u1);  u+ = 1/3 u + 2/3 E(u2)
 * Each stage refreshes the halo from its own input.  The intermediate states
 * u1, u2 are the storage of intermediate results across multiple update steps
 * that the paper's Limitations paragraph (Sec. 5) says LOPe does not provide:
 * the trapezoid path keeps them in shared memory, the TMA and direct paths in
 * the work buffers.  nsteps of lope_apply then counts Runge-Kutta steps.
 * Not supported by lope_apply_batch and the adjoint calls (UNSUPPORTED).
 * Errors: LOPE_ERR_INVALID for an unknown scheme. */
typedef enum { LOPE_SCHEME_EULER = 1, LOPE_SCHEME_RK2 = 2, LOPE_SCHEME_RK3 = 3 } lope_scheme;
lope_status lope_stencil_set_scheme(lope_stencil* stencil, lope_scheme scheme);

/* Number of grid states each work buffer of lope_apply must hold for this
 * stencil's scheme: 2 for RK3 (both stage states, the second directly after
 * the first), else 1. */
lope_status lope_work_states(const lope_stencil* stencil, int* states);

/* Apply the local function at every interior point, nsteps times (Sec. 3.2:
 * each do-concurrent sweep is followed by a halo refresh).  Every sweep reads
 * a frozen snapshot of the previous state (Sec. 2.2 double buffering, Sec. 3.5
 * implicit synchronisation): results do not depend on tiling, traversal order
 * or temporal blocking.
 *   in[nfields]   read-only input state (never written)
 *   out[nfields]  final state; must not alias in
 *   work[nfields] scratch state of the same size (lope_work_states() states
 *                 for multi-stage schemes), needed when nsteps >= 2 or the
 *                 scheme has several stages (may be NULL for Euler, nsteps <= 1)
 * nsteps = 0 copies in to out.  The planner picks kernel, tile and temporal
 * depth (see lope_apply_with).  Errors: LOPE_ERR_INVALID (aliasing, NULL,
 * misaligned pointers, stencil radius above the declared halo, dimension
 * mismatch), LOPE_ERR_UNSUPPORTED (dtype/stencil pair not built),
 * LOPE_ERR_CUDA (launch failure). */
lope_status lope_apply(const lope_grid* grid, const lope_stencil* stencil, const void* const* in,
                       void* const* out, void* const* work, int64_t nsteps, void* cuda_stream);

/* The end-to-end form of lope_apply for a state held in host memory: copies
 * host_in[nfields] to the device buffers dev_in, runs lope_apply(dev_in ->
 * dev_out, dev_work as the work buffers), and copies dev_out back to
 * host_out[nfields], all in order on the stream (asynchronous).  dev_in is
 * overwritten with the input; the other conventions are lope_apply's.  Host
 * buffers should be page-locked (cudaHostAlloc / pinned) for asynchronous,
 * full-bandwidth copies; pageable host memory works but the copies then
 * synchronise.  Several calls on different streams with their own device
 * buffers overlap one call's copies with another's sweeps. */
lope_status lope_apply_host(const lope_grid* grid, const lope_stencil* stencil,
                            const void* const* host_in, void* const* host_out,
                            void* const* dev_in, void* const* dev_out, void* const* dev_work,
                            int64_t nsteps, void* cuda_stream);

/* Launch choices, for tests and tuning.  Zero fields mean "planner decides".
 *   path:    0 auto;
 *            1 TMA tiles (2D tiles, any stencil / 3D z-march, star stencils;
 *              16-byte row pitch);
 *            2 shared-memory trapezoid tiles with temporal blocking (2D, any
 *              stencil, any shape);
 *            3 direct (any stencil, one thread per point);
 *            4 plane march (3D, any stencil and row pitch; not for the
 *              adjoint; source stencils only as one-field star functions with
 *              FP32 / FP64 storage and plain sweeps): tiles marched along z
 *              through a shared-memory ring of planes.  FP32 / FP64 star
 *              functions: 64 x 64 tiles (32 x 32 for FP64; tile_y = 1 for a
 *              builtin: 64 x 32 / 32 x 32) whose planes producer warps copy in;
 *              box functions and multi-stage steps: 64 x 16 tiles; BF16:
 *              64 x 4 tiles.
 *            For grids whose row pitch is not a multiple of 16 bytes the
 *            planner takes trapezoid tiles fusing 4 sweeps in 2D (128 x 32
 *            for one field, 64 x 16 for several) and the plane march in 3D.
 *   tile_x, tile_y: tile shape for path 2 (tile_x in {32,64,128}, tile_y in
 *            {8,16,32}); for path 1, tile_y = 1 or 2 forces the short or the
 *            tall tiles (0: tall from 2^22 points in 2D, 2^26 in 3D).
 *   tsteps:  temporal depth k (sweeps fused per launch; path 2 only, 1..8).
 *   graph:   0 auto, 1 capture the launch sequence in a CUDA graph, -1 never. */
typedef struct {
  int path;
  int tile_x, tile_y;
  int tsteps;
  int graph;
} lope_launch;

lope_status lope_apply_with(const lope_grid* grid, const lope_stencil* stencil,
                            const void* const* in, void* const* out, void* const* work,
                            int64_t nsteps, const lope_launch* cfg, void* cuda_stream);

/* The plan lope_apply_with would run for these arguments, without running
 * it: *plan receives the launch path, tile, temporal depth and whether the
 * launch sequence is replayed from a CUDA graph (1) or not (-1), and
 * *launches (may be NULL) the number of kernel launches.  Host only: no CUDA
 * call is made, so it also works on a machine without a GPU.  Pointers are
 * checked (alignment, aliasing, work buffers) but never dereferenced.
 * Errors: those of lope_apply_with's argument checks; LOPE_ERR_INVALID for a
 * NULL plan. */
lope_status lope_plan(const lope_grid* grid, const lope_stencil* stencil, const void* const* in,
                      void* const* out, void* const* work, int64_t nsteps, const lope_launch* cfg,
                      lope_launch* plan, int64_t* launches);

/* Time candidate launch choices on the caller's buffers (out and work are
 * overwritten) and remember the fastest for this grid shape, dtype, stencil and
 * boundary; later lope_apply calls use it.  *best receives the choice and
 * *best_ms its time for nsteps.  Synchronises the stream. */
lope_status lope_autotune(const lope_grid* grid, const lope_stencil* stencil,
                          const void* const* in, void* const* out, void* const* work,
                          int64_t nsteps, lope_launch* best, double* best_ms, void* cuda_stream);

/* Autotune cache file.  lope_tune_cache_save writes every choice that
 * lope_autotune and lope_autotune_batch made in this process (builtin and
 * weight-table stencils; source stencils are left out) to the text file at
 * path, one entry per line, tagged with a GPU name: gpu_name, or the current
 * device's name when gpu_name is NULL.  lope_tune_cache_load installs the
 * entries of such a file whose GPU name matches, so that later lope_apply and
 * lope_apply_batch calls plan with them; lines that do not parse or name
 * another GPU are skipped, and *loaded (may be NULL) receives the number
 * installed.  A remembered choice that cannot run a grid (e.g. a TMA plan for
 * a misaligned input) is ignored at planning time.  The paper has no
 * counterpart; this is a property of the library only.
 * Errors: LOPE_ERR_INVALID for a NULL path or a file that cannot be opened or
 * written; LOPE_ERR_CUDA when gpu_name is NULL and no device can be queried. */
lope_status lope_tune_cache_save(const char* path, const char* gpu_name);
lope_status lope_tune_cache_load(const char* path, const char* gpu_name, int* loaded);

/* Batched form: n independent grids of possibly different extents and
 * boundaries (same dtype, nfields and stencil) advanced nsteps each in one
 * persistent launch per call, replayed from a cached CUDA graph.  in/out/work
 * hold n*nfields pointers, grid-major.  workspace is caller device memory of at
 * least lope_batch_workspace_size bytes (about 64 bytes per 64 x 64 tile of
 * the batch, plus the grid list); it holds the work list, the tile records,
 * the tile-claim counter and the inter-block barrier, and must stay untouched
 * between calls that reuse it.
 * cfg may be NULL: the choice of the batch autotuner for this batch (see
 * lope_autotune_batch), else, for FP32 star functions of radius 1-2 (jacobi5,
 * star9r2, linear star tables), the two-sweep register tiles (cfg->path 1:
 * 64 x 64 tiles staged by plain loads, any row pitch, two sweeps per pass),
 * and the trapezoid tiles otherwise (cfg->path 2: 64 x 32 tiles, depth 4;
 * tile_x, tile_y and tsteps choose another shape and depth).  Errors as
 * lope_apply; LOPE_ERR_TIMEOUT is reported by lope_sync_status if a bounded
 * barrier wait gave up. */
lope_status lope_batch_workspace_size(int n, const lope_grid* const* grids,
                                      const lope_stencil* stencil, const lope_launch* cfg,
                                      size_t* bytes);
lope_status lope_apply_batch(int n, const lope_grid* const* grids, const lope_stencil* stencil,
                             const void* const* in, void* const* out, void* const* work,
                             int64_t nsteps, const lope_launch* cfg, void* workspace,
                             size_t workspace_bytes, void* cuda_stream);

/* Batch autotuner: times the batched launch over the two-sweep register tiles
 * (where they apply) and the trapezoid tiles of shapes {128, 64} x {32, 16}
 * and temporal depths {1, 2, 4, 5} on the caller's buffers (out and work
 * are overwritten), stores the fastest for this batch (grid extents and
 * boundaries, dtype, stencil) and returns it in *best (*best_ms its time for
 * nsteps).  Later lope_apply_batch calls with cfg NULL (or zero tile/depth) on
 * a batch with the same signature use it.  Synchronises the stream. */
lope_status lope_autotune_batch(int n, const lope_grid* const* grids, const lope_stencil* stencil,
                                const void* const* in, void* const* out, void* const* work,
                                int64_t nsteps, void* workspace, size_t workspace_bytes,
                                lope_launch* best, double* best_ms, void* cuda_stream);

/* Differentiation of u_T = A^T u_0 for linear stencils, by the discrete adjoint
 * (transposed stencil, run backward in time) with recomputation from
 * checkpoints stored every `checkpoint_every` steps.
 *
 * lope_adjoint: loss = sum (u_T - target)^2 (FP64 accumulation), then
 *   grad_u0 = dL/du_0 (device, grid dtype) and *grad_coeff = dL/dc (host,
 *   diffusion-form builtins only; 0 otherwise) and *loss (host).  Synchronises.
 * lope_vjp: the same reverse sweep for an arbitrary upstream gradient grad_uT
 *   (device); *grad_coeff_dev is a device double that receives dL/dc (may be
 *   NULL).  Asynchronous.
 * lope_forward_ckpt: the forward pass alone, writing u_T and leaving the
 *   checkpoints in the workspace for a later lope_vjp with the same u0,
 *   nsteps and checkpoint_every (vjp then skips its own forward when
 *   reuse_checkpoints = 1).
 * workspace: device memory of lope_workspace_size(grid, stencil, nsteps,
 *   checkpoint_every) bytes.  Errors: LOPE_ERR_UNSUPPORTED for non-linear
 *   stencils; LOPE_ERR_ALLOC if workspace_bytes is too small. */
lope_status lope_workspace_size(const lope_grid* grid, const lope_stencil* stencil,
                                int64_t nsteps, int64_t checkpoint_every, size_t* bytes);
lope_status lope_forward_ckpt(const lope_grid* grid, const lope_stencil* stencil, const void* u0,
                              void* uT, int64_t nsteps, int64_t checkpoint_every, void* workspace,
                              size_t workspace_bytes, void* cuda_stream);
lope_status lope_vjp(const lope_grid* grid, const lope_stencil* stencil, const void* u0,
                     const void* grad_uT, int64_t nsteps, int64_t checkpoint_every,
                     int reuse_checkpoints, void* grad_u0, double* grad_coeff_dev,
                     void* workspace, size_t workspace_bytes, void* cuda_stream);
lope_status lope_adjoint(const lope_grid* grid, const lope_stencil* stencil, const void* u0,
                         const void* target, int64_t nsteps, int64_t checkpoint_every,
                         void* grad_u0, double* grad_coeff, double* loss, void* workspace,
                         size_t workspace_bytes, void* cuda_stream);

/* FP64 reductions over a stored field (conservation checks, losses):
 * *result_dev (device double) = sum x[i]  (op 0), or sum (x[i]-y[i])^2 (op 1),
 * over n elements of dtype `dtype`.  scratch is device memory of at least
 * lope_reduce_scratch_bytes() bytes for per-block partial sums; the summation
 * order is fixed, so results are reproducible run to run. */
size_t lope_reduce_scratch_bytes(void);
lope_status lope_reduce(int op, lope_dtype dtype, const void* x, const void* y, int64_t n,
                        double* result_dev, void* scratch, void* cuda_stream);

/* Runtime options (process-wide):
 *   "wait_limit_ms"      limit of each bounded inter-block barrier wait in the
 *                        batched kernel (default 1000).
 *   "batch_skip_arrive"  failure-detection hook for tests: block `value` of the
 *                        next batched plans never arrives at the first
 *                        inter-block barrier, so the other blocks' bounded waits
 *                        run out and lope_sync_status reports LOPE_ERR_TIMEOUT
 *                        (-1, the default, disables it).  No fault is raised on
 *                        the GPU: every wait ends by itself.
 *   "fail_alloc"         fault injection on the host: the next `value` calls
 *                        that may allocate library-owned memory (the
 *                        per-device state of the first apply, a new batch
 *                        plan) fail with LOPE_ERR_ALLOC before any CUDA call;
 *                        0 (the default) disables it.
 *   "log"                1: print each distinct plan that lope_apply and
 *                        lope_apply_with resolve, once, as one line on stderr
 *                        (grid, boundaries, local function, scheme, path, tile,
 *                        depth, launch count, graph); 0: silent.  The initial
 *                        value is that of the LOPE_LOG environment variable
 *                        (unset: 0).
 * Errors: LOPE_ERR_INVALID for an unknown name or out-of-range value. */
lope_status lope_set_option(const char* name, int64_t value);

/* The FP64 reduction of lope_reduce without any memory from the caller or
 * the allocator: for callers that cannot provide scratch memory, such as code
 * whose device memory is entirely owned by another allocator, or loops where
 * an allocation call (which may synchronise the device) is not acceptable.
 * The paper has no counterpart; this is a property of the library only.
 * The per-block partial sums live in a 512 KiB array that is part of the
 * library image (held on every GPU that loads the library until the process
 * exits).  n must not exceed 2^28 elements (LOPE_ERR_INVALID otherwise).
 * The first call on a device looks up the array's device address, once, and
 * keeps it for the life of the process; make that first call before any
 * stream capture.  A device reset (cudaDeviceReset) unloads the array, so the
 * kept address is no longer valid: do not call this entry point on a device
 * after resetting it in the same process.  All calls on a device share the
 * array, so calls that overlap on the GPU race: order them on one stream or
 * synchronise between them.  Every element of the array that a call reads was
 * written earlier in that call, so results never depend on previous calls.
 * Arguments and result as lope_reduce. */
lope_status lope_reduce_noalloc(int op, lope_dtype dtype, const void* x, const void* y, int64_t n,
                                double* result_dev, void* cuda_stream);

/* Synchronise the stream, then report (and clear) the device-side error flag:
 * LOPE_ERR_TIMEOUT if a bounded wait gave up, LOPE_ERR_INVALID if a run-time
 * compiled local function read outside its declared halo, else LOPE_OK. */
lope_status lope_sync_status(void* cuda_stream);

/* Number of kernels this library has launched in this process (graph
 * replays count each kernel node once per replay). */
int64_t lope_launch_count(void);

/* Message for the last failed call on this thread (never NULL). */
const char* lope_last_error(void);

/* Library version string. */
const char* lope_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LOPE_H */
