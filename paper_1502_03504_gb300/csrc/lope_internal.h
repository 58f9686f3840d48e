// Internal types shared by the host planner (api.cu) and the kernel files.
// The part outside the host-only sections also compiles under NVRTC, for
// run-time compiled local functions (jit.cu).
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "lope.h"
#endif

namespace lope {

// Stencil kinds (builtin names of lope_stencil_create_builtin).
enum : int { kLinear = 0, kJacobi5 = 1, kDiff7 = 2, kStar9r2 = 3, kSwe = 4, kSweFlux = 5, kUser = 6 };
constexpr int kUserParams = 8;  // parameters P[0..7] of a user-written local function
enum : int { kF64 = 0, kF32 = 1, kBF16 = 2 };
// Boundary kinds of one side of an axis.  kExternal (slowest axis only): the
// halo is read from the input buffer beyond the grid, where the caller keeps
// the neighbouring slab's planes (or rows) -- the destination of a halo
// exchange between the slabs of a decomposed grid.
enum : int { kPeriodic = 0, kDirichlet = 1, kExternal = 2 };
enum : int { kPathAuto = 0, kPathTma = 1, kPathTrap = 2, kPathDirect = 3, kPathMarch = 4 };

// Device error codes written to the error flag.
constexpr int kErrTimeout = 1;
constexpr int kErrHalo = 2;  // a run-time compiled function read beyond its declared halo
// Upper bound of any single in-kernel wait (ns).  Normal waits last
// microseconds; this only ends a wait that can no longer succeed.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

constexpr int kMaxFields = 3;
constexpr int kMaxRadius = 2;

// A grid as the kernels see it.  Axes are stored slowest first and always as
// three: a 2D grid has n[0] = 1.
struct Geom {
  int ndim;
  int64_t n[3];
  int bc[3][2];
  double bval[3][2];
  int dtype;
  int nf;
};

struct StencilDesc {
  int kind;
  int ndim;
  int radius;
  int stages;          // time-stepping scheme: 1 forward Euler (the function itself), 2 / 3 SSP-RK
  bool star;           // only axis-aligned taps
  double prm[4];       // c | dt, g, H | dt, g, f, H
  double box[125];     // (2r+1)^ndim weight table, slowest offset first
  double star_w[3][2 * kMaxRadius + 1];  // per axis (0 = x, 1 = y, 2 = z), centre in [0][r]
  int user_nf;         // kUser: number of fields
  void* jit;           // kUser: the run-time compiled program (host object, jit.cu)
};

// Coefficients (a, b) of stage s (1-based, s >= 2) of the strong-stability-
// preserving Runge-Kutta schemes (Shu and Osher, 1988) with `stages` stages,
// written as convex combinations of forward-Euler steps:
//   RK2: u1 = E(u); u+ = 1/2 u + 1/2 E(u1)
//   RK3: u1 = E(u); u2 = 3/4 u + 1/4 E(u1); u+ = 1/3 u + 2/3 E(u2)
// Stage 1 is E itself (a = 0, b = 1).
__host__ __device__ inline void rk_coeffs(int stages, int s, double* a, double* b) {
  if (stages == 2) {
    *a = 0.5;
    *b = 0.5;
  } else if (s == 2) {
    *a = 0.75;
    *b = 0.25;
  } else {
    *a = 1.0 / 3.0;
    *b = 2.0 / 3.0;
  }
}

#ifndef __CUDACC_RTC__
// One launch: `ksteps` sweeps from in to out.
struct StepArgs {
  Geom g;
  StencilDesc s;
  const void* in[kMaxFields];
  void* out[kMaxFields];
  int ksteps;
  int tile_x, tile_y;
  bool adjoint;          // run the transposed stencil (lambda halo: Dirichlet -> 0)
  const void* ut;        // adjoint: state u_t read at the local element
  const void* base[kMaxFields];  // RK stage >= 2: state at the start of the step
  double rk_a, rk_b;     // RK stage >= 2: out = rk_a * base + rk_b * E(in)
  int stage;             // RK: 0/1 plain sweep of E; >= 2 combining stage (TMA/direct)
  double* partials;      // adjoint: per-block FP64 partial sums (accumulated)
  int partial_count;     // adjoint: number of partial slots available
  int* err;              // device error flag
  cudaStream_t stream;
};

// Launchers (each returns the number of blocks it used through *blocks when
// non-NULL, so that the adjoint can size its partial-sum buffer).
cudaError_t launch_tma(const StepArgs& a, int* blocks);
cudaError_t launch_tma_stage(const StepArgs& a);  // a.stage >= 2 (k_tma_stage.cu)
bool tma_supported(const StepArgs& a);
cudaError_t launch_trap2d(const StepArgs& a);
bool trap2d_supported(const StepArgs& a);
cudaError_t launch_direct(const StepArgs& a, int* blocks);
// 3D plane march for grids the TMA tiles cannot stage (not for the adjoint;
// run-time compiled functions: one-field star functions, FP32 / FP64, plain
// sweeps).
cudaError_t launch_march(const StepArgs& a);
bool march_supported(const StepArgs& a);
// Run-time compiled local functions (jit.cu).
struct JitProgram;
lope_status jit_create(const char* body, int ndim, int radius, int nf, bool star,
                       const double* prm, int nprm, JitProgram** out);
void jit_destroy(JitProgram* jp);
lope_status jit_compile(JitProgram* jp, int dtype, std::string* err);
bool jit_tma_ok(const JitProgram* jp);
// Launch one sweep / stage of a kUser stencil on path kPathTma, kPathTrap,
// kPathMarch or kPathDirect (a.stage >= 2: combining Runge-Kutta stage; a.s.stages >= 2 on
// the trapezoid: fused steps).
cudaError_t jit_launch(const StepArgs& a, int path);

// Multi-stage forms on the generic kernels (k_generic_rk.cu): fused trapezoid
// steps (kGenTrap), or a combining stage on the direct kernel (kGenDirect) or
// the plane march (kGenMarch).
enum : int { kGenDirect = 0, kGenTrap = 1, kGenMarch = 2 };
cudaError_t launch_generic_rk(const StepArgs& a, int kind, int* blocks);
bool direct_supported(const StepArgs& a);
bool has_external(const Geom& g);
int tma_blocks(const StepArgs& a);
int direct_blocks(const StepArgs& a);

// Reductions (k_reduce.cu).
constexpr int kReduceBlocks = 608;  // 4 x 152 SMs; partial sums per reduction
cudaError_t launch_reduce(int op, int dtype, const void* x, const void* y, int64_t n,
                          double* partials, double* result, cudaStream_t s);
cudaError_t launch_loss_seed(int dtype, const void* uT, const void* target, void* lam, int64_t n,
                             double* partials, double* loss, cudaStream_t s);
cudaError_t launch_finalize(const double* partials, int count, double* result, int accumulate,
                            cudaStream_t s);

// Batched persistent kernel (k_batch.cu).
struct BatchGrid {
  const void* in;
  void* out;
  void* work;
  int nx, ny;
  int bc[2][2];       // [axis: 0 = y, 1 = x][side]
  double bval[2][2];
  int tiles_x;
  int first_item;     // index of this grid's first tile in the global item list
};
// One tile of the two-sweep batched tiles (mode 1), 64 bytes: everything a
// block needs to stage and sweep it, read with four 16-byte loads.  Filled
// on the device from the grid list at the start of each batched launch.
struct __align__(16) BatchItem {
  const float* in;
  float* out;
  float* work;
  int nx, ny, x0, y0;
  int bc;             // side kinds, 8 bits each: y low, y high, x low, x high
  float vy0, vy1, vx0, vx1;
  int pad;
};
struct BatchPlanDev {
  const BatchGrid* grids;  // device
  BatchItem* items;        // device, one per tile (mode 1 only)
  int ngrids;
  int nitems;
  int tile_x, tile_y;
  int ksteps;
  int64_t nsteps;
  unsigned int* barrier;   // device counter, zeroed before each launch
  unsigned long long* claim;  // device tile-claim counter, zeroed before each launch
  int* err;
  unsigned long long wait_ns;  // limit of each barrier wait
  int skip_block;              // test hook: this block skips its first arrival (-1: none)
  int mode;                    // 0: trapezoid tiles (k sweeps per pass); 1: two-sweep
                               // register tiles (64 x 64, two sweeps per pass)
};
cudaError_t launch_batch(const BatchPlanDev& p, const StencilDesc& s, int dtype, int blocks,
                         cudaStream_t st);
int batch_max_blocks(const StencilDesc& s, int dtype, int tile_x, int tile_y, int ksteps,
                     int mode = 0);
// Tile of the two-sweep batched tiles (mode 1).
constexpr int kBatchTb2X = 64, kBatchTb2Y = 64;
size_t trap_smem_bytes(int dtype, int nf, int tile_x, int tile_y, int halo, int stages = 1);

void count_launches(int64_t n);

#endif  // __CUDACC_RTC__

}  // namespace lope

#ifndef __CUDACC_RTC__
// Record the last-error message of the calling thread (defined in api.cu).
lope_status lope_fail_external(lope_status st, const char* msg);
#endif
