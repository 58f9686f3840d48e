// C ABI of the LOPe library: handles, validation, the launch planner (kernel
// path, tile shape, temporal depth), CUDA-graph caching, the autotuner, the
// batched-plan cache and the adjoint driver with checkpointed recomputation.
//
// Halo declarations and the no-out-of-bounds rule (Sec. 2.2 "Halo regions",
// Sec. 3.5) are checked here: a stencil may not read further than the halo
// its grid declares.  There is no host fallback: every computation runs in
// the kernels of this library.
#include <algorithm>
#include <cctype>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <initializer_list>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "lope.h"
#include "lope_internal.h"

struct lope_grid {
  lope::Geom g;
  int halo_lo[3], halo_hi[3];  // per axis, slowest first (2D: axis 0 unused)
};

struct lope_stencil {
  lope::StencilDesc s;
  int nf;
  lope::JitProgram* jit;  // user-written local functions (owned)
};

namespace lope {

namespace {

thread_local std::string g_last_error = "no error";
std::atomic<int64_t> g_wait_limit_ms{1000};
std::atomic<int64_t> g_skip_arrive{-1};
// Fault injection on the host: the next g_fail_alloc calls that may allocate
// library-owned memory fail with LOPE_ERR_ALLOC before touching CUDA.
std::atomic<int64_t> g_fail_alloc{0};

bool take_alloc_failure() {
  int64_t v = g_fail_alloc.load();
  while (v > 0)
    if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return true;
  return false;
}
thread_local bool g_capturing = false;
thread_local int64_t g_captured = 0;  // kernels recorded by the capture in progress
std::atomic<int64_t> g_launches{0};

lope_status fail(lope_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

lope_status cuda_fail(cudaError_t e, const char* what) {
  return fail(LOPE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int esize(int dtype) { return dtype == kF64 ? 8 : dtype == kF32 ? 4 : 2; }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int64_t npts(const Geom& g) { return g.n[0] * g.n[1] * g.n[2]; }

// Per-device state: the device error flag and a stream used for graph capture.
struct DevState {
  int* err = nullptr;
  cudaStream_t capture = nullptr;
};
std::mutex g_dev_mu;
std::map<int, DevState> g_dev;

lope_status dev_state(DevState** out) {
  if (take_alloc_failure()) return fail(LOPE_ERR_ALLOC, "allocation refused (fail_alloc option)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DevState& d = g_dev[dev];
  if (!d.err) {
    if ((e = cudaMalloc(&d.err, sizeof(int))) != cudaSuccess) return cuda_fail(e, "cudaMalloc(error flag)");
    if ((e = cudaMemset(d.err, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "cudaMemset");
    if ((e = cudaStreamCreateWithFlags(&d.capture, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamCreate");
  }
  *out = &d;
  return LOPE_OK;
}

// ------------------------------------------------------------------ validation
int stencil_nf(const StencilDesc& s) {
  if (s.kind == kUser) return s.user_nf;
  return (s.kind == kSwe || s.kind == kSweFlux) ? 3 : 1;
}

lope_status check_pair(const lope_grid* grid, const lope_stencil* st) {
  if (!grid || !st) return fail(LOPE_ERR_INVALID, "NULL grid or stencil");
  const Geom& g = grid->g;
  const StencilDesc& s = st->s;
  if (s.ndim != g.ndim) return fail(LOPE_ERR_INVALID, "stencil and grid dimensions differ");
  if (stencil_nf(s) != g.nf) return fail(LOPE_ERR_INVALID, "stencil and grid field counts differ");
  for (int ax = 3 - g.ndim; ax < 3; ++ax) {
    if (s.radius > grid->halo_lo[ax] || s.radius > grid->halo_hi[ax])
      return fail(LOPE_ERR_INVALID, "stencil radius exceeds the declared halo (out-of-bounds read)");
    if (g.bc[ax][0] == kPeriodic && g.n[ax] < s.radius)
      return fail(LOPE_ERR_INVALID, "periodic axis shorter than the stencil radius");
  }
  return LOPE_OK;
}

// States each work buffer holds: two for the RK3 stage sequence (u1, u2), one
// otherwise.
int work_states(const StencilDesc& s) { return s.stages == 3 ? 2 : 1; }

// Bytes of the caller's buffer an input reads beyond the grid on its external
// sides (radius planes / rows each), before and after the grid.
void external_pads(const Geom& g, int radius, size_t* before, size_t* after) {
  const int sax = 3 - g.ndim;
  const size_t slice = size_t(npts(g) / g.n[sax]) * esize(g.dtype);
  *before = g.bc[sax][0] == kExternal ? size_t(radius) * slice : 0;
  *after = g.bc[sax][1] == kExternal ? size_t(radius) * slice : 0;
}

lope_status check_fields(const Geom& g, const void* const* in, void* const* out, void* const* work,
                         bool need_work, int wstates = 1, int radius = 0) {
  if (!in || !out) return fail(LOPE_ERR_INVALID, "NULL field array");
  if (need_work && !work) return fail(LOPE_ERR_INVALID, "nsteps >= 2 needs work buffers");
  size_t pad_lo = 0, pad_hi = 0;
  external_pads(g, radius, &pad_lo, &pad_hi);
  for (int f = 0; f < g.nf; ++f) {
    if (!in[f] || !out[f]) return fail(LOPE_ERR_INVALID, "NULL field pointer");
    if (!aligned16(in[f]) || !aligned16(out[f])) return fail(LOPE_ERR_INVALID, "field pointer not 16-byte aligned");
    if (need_work && (!work[f] || !aligned16(work[f]))) return fail(LOPE_ERR_INVALID, "bad work pointer");
    const size_t bytes = size_t(npts(g)) * esize(g.dtype);
    auto overlap = [&](const void* a, size_t na, const void* b, size_t nb) {
      const char* x = static_cast<const char*>(a);
      const char* y = static_cast<const char*>(b);
      return x < y + nb && y < x + na;
    };
    const size_t wbytes = bytes * size_t(wstates);
    // the input as read: the grid and its external halo planes
    const void* in_read = static_cast<const char*>(in[f]) - pad_lo;
    const size_t in_bytes = bytes + pad_lo + pad_hi;
    for (int h = 0; h < g.nf; ++h) {
      if (overlap(in_read, in_bytes, out[h], bytes))
        return fail(LOPE_ERR_INVALID, "out aliases in (double buffering required)");
      if (need_work && (overlap(work[f], wbytes, out[h], bytes) || overlap(work[f], wbytes, in[h], bytes)))
        return fail(LOPE_ERR_INVALID, "work aliases in or out");
      if (need_work && h != f && overlap(work[f], wbytes, work[h], wbytes))
        return fail(LOPE_ERR_INVALID, "work buffers of two fields overlap");
    }
  }
  return LOPE_OK;
}

// ------------------------------------------------------------------ planning
struct Choice {
  int path, tile_x, tile_y, k;
};

using TuneKey = std::tuple<int, int64_t, int64_t, int64_t, int, int, int, int, int, int, int, int64_t>;
std::mutex g_tune_mu;
std::map<TuneKey, Choice> g_tune;

TuneKey tune_key(const Geom& g, const StencilDesc& s) {
  int bcs = 0, ext = 0;
  for (int ax = 0; ax < 3; ++ax)
    for (int sd = 0; sd < 2; ++sd) {
      bcs = bcs * 2 + (g.bc[ax][sd] == kDirichlet);
      ext = ext * 2 + (g.bc[ax][sd] == kExternal);
    }
  bcs |= ext << 6;
  return TuneKey(g.ndim, g.n[0], g.n[1], g.n[2], g.dtype, s.kind, s.radius, int(s.star), bcs,
                 g.nf, s.stages, int64_t(reinterpret_cast<uintptr_t>(s.jit)));
}

StepArgs base_args(const Geom& g, const StencilDesc& s, int* err, cudaStream_t st) {
  StepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = g;
  a.s = s;
  a.ksteps = 1;
  a.err = err;
  a.stream = st;
  return a;
}

// Whether launch choice c can run this grid and stencil (a.in holds the
// input pointers, whose alignment the TMA path checks).
bool choice_supported(StepArgs a, const Choice& c) {
  a.ksteps = c.k;
  a.tile_x = c.tile_x;
  a.tile_y = c.tile_y;
  bool ok = false;
  switch (c.path) {
    case kPathTma: ok = tma_supported(a); break;
    case kPathTrap: ok = trap2d_supported(a); break;
    case kPathDirect: ok = direct_supported(a); break;
    case kPathMarch: ok = march_supported(a); break;
    default: ok = false;
  }
  return ok && !(a.s.stages >= 2 && c.path != kPathTrap && c.k != 1);
}

Choice default_choice(const Geom& g, const StencilDesc& s, int* err) {
  StepArgs a = base_args(g, s, err, nullptr);
  for (int f = 0; f < g.nf; ++f) a.in[f] = reinterpret_cast<const void*>(uintptr_t(256));
  {
    // a remembered autotuner choice (possibly loaded from a cache file) is
    // used when it can run this grid
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(g, s));
    if (it != g_tune.end() && choice_supported(a, it->second)) return it->second;
  }
  if (s.stages >= 2 && g.ndim == 2 && g.nf == 1 && g.dtype == kF32) {
    // Multi-stage steps of a single FP32 field: the fused trapezoid keeps the
    // stage states on chip (one read and one write per step instead of one
    // per stage) and measured 1.3x faster than one TMA launch per stage for
    // the 5-point diffusion at 8192^2.  For several fields or BF16 storage the
    // per-stage TMA launches measured as fast or faster (Gray-Scott, shallow
    // water), so those take the default below.
    a.tile_x = 128;
    a.tile_y = 16;
    if (trap2d_supported(a)) return {kPathTrap, 128, 16, 1};
  }
  if (g.ndim == 2 && s.stages == 1 &&
      size_t(npts(g)) * esize(g.dtype) * size_t(g.nf) <= (size_t(8) << 20)) {
    // A state that stays in L2 makes each sweep a short, launch-bound kernel:
    // fuse 4 sweeps per launch in trapezoid tiles (measured on GB300 for a
    // 256^2 FP64 grid, 100 steps: 0.44 ms against 0.56 ms for one TMA sweep
    // per launch).
    a.tile_x = 64;
    a.tile_y = 16;
    a.ksteps = 4;
    if (trap2d_supported(a)) return {kPathTrap, 64, 16, 4};
    a.ksteps = 1;
  }
  if (s.stages == 1 && ((g.ndim == 3 && npts(g) >= (int64_t(1) << 21)) ||
                         (g.ndim == 2 && npts(g) >= (int64_t(1) << 22)))) {
    // Two sweeps per launch halve the HBM bytes per sweep.  Measured on
    // GB300, 50 sweeps (one sweep per launch -> two):
    //   3D diff7 FP32 Dirichlet 0: 512^3 9.10 -> 5.46 ms, 384^3 3.82 -> 2.58,
    //   256^3 1.05 -> 0.89, 128^3 0.32 -> 0.27; BF16 512^3 6.67 -> 6.22,
    //   256^3 1.04 -> 0.94 (its one-sweep march is far from the copy peak
    //   already and the two-sweep march is bound by instruction issue);
    //   2D star9r2 FP32 8192^2 periodic 4.26 -> 3.25 ms, Dirichlet 4.14 ->
    //   3.05; jacobi5 FP32 8192^2 4.13 -> 2.84 / 4.21 -> 2.63; BF16 8192^2
    //   star9r2 3.71 -> 3.47, jacobi5 about equal; 4096^2 FP32 1.2-1.45x;
    //   linear shallow water 4096^2 x3 x200 FP32 14.97 -> 7.82 ms, BF16
    //   7.60 -> 7.18; nonlinear shallow water (box halo) FP32 per sweep
    //   74.8 -> 56.4 us.  BF16 box functions stay at one sweep per launch:
    //   their two-sweep tiles are bound by instruction issue (nonlinear
    //   shallow water 47.1 -> 59.2 us per sweep).
    a.ksteps = 2;
    if (!(g.ndim == 2 && g.dtype == kBF16 && !s.star) && tma_supported(a))
      return {kPathTma, 0, 0, 2};
    a.ksteps = 1;
  }
  if (tma_supported(a)) return {kPathTma, 0, 0, 1};
  if (has_external(g)) return {kPathDirect, 0, 0, 1};
  if (g.ndim == 2) {
    // Rows whose pitch is not a multiple of 16 bytes cannot be TMA-staged.
    // Trapezoid tiles fusing 4 sweeps measured 2.4x faster than one sweep per
    // launch (FP32, 20 steps): jacobi5 7094^2 2.01 ms on 128 x 32 tiles
    // against 4.85 ms on 64 x 32 tiles with k = 1; the three-field swe_flux
    // 6.6 ms on 64 x 16 tiles against 14.8 ms (and 18.3 ms on 128 x 32 tiles,
    // whose shared memory leaves one block per SM).
    a.tile_x = g.nf == 1 ? 128 : 64;
    a.tile_y = g.nf == 1 ? 32 : 16;
    a.ksteps = 4;
    if (s.stages == 1 && trap2d_supported(a)) return {kPathTrap, a.tile_x, a.tile_y, 4};
    return {kPathTrap, 64, 32, 1};
  }
  // 3D rows that cannot be TMA-staged: the plane march (diff7 FP32
  // 130 x 500 x 510: 75.5 us per sweep on the copied-plane z-march against
  // 232 us on the direct kernel), else the direct kernel (the adjoint, and
  // run-time compiled functions of several fields, box functions, BF16 storage
  // or multi-stage steps).
  a.ksteps = 1;
  if (march_supported(a)) return {kPathMarch, 0, 0, 1};
  return {kPathDirect, 0, 0, 1};
}

lope_status resolve(const Geom& g, const StencilDesc& s, const void* const* in,
                    const lope_launch* cfg, int* err, Choice* c) {
  Choice d = default_choice(g, s, err);
  if (cfg && cfg->path != kPathAuto) {
    d.path = cfg->path;
    d.tile_x = cfg->tile_x;
    d.tile_y = cfg->tile_y;
    d.k = cfg->tsteps > 0 ? cfg->tsteps : 1;
  } else if (cfg) {
    if (cfg->tsteps > 0) d.k = cfg->tsteps;
    if (cfg->tile_x > 0) d.tile_x = cfg->tile_x;
    if (cfg->tile_y > 0) d.tile_y = cfg->tile_y;
  }
  if (d.path == kPathTrap) {
    if (d.tile_x <= 0) d.tile_x = 64;
    if (d.tile_y <= 0) d.tile_y = 32;
  }
  StepArgs a = base_args(g, s, err, nullptr);
  for (int f = 0; f < g.nf; ++f) a.in[f] = in ? in[f] : nullptr;
  if (!choice_supported(a, d)) return fail(LOPE_ERR_UNSUPPORTED, "requested launch path does not support this grid/stencil/depth");
  *c = d;
  return LOPE_OK;
}

// Plan log: with option "log" = 1 (initially the value of the LOPE_LOG
// environment variable), every distinct plan an apply call resolves is printed
// once on stderr: the grid, the local function and the launch sequence.
std::atomic<int> g_log{-1};
std::mutex g_log_mu;
std::set<std::vector<int64_t>> g_logged;

bool log_enabled() {
  int v = g_log.load();
  if (v < 0) {
    const char* e = std::getenv("LOPE_LOG");
    v = (e && std::atoi(e) > 0) ? 1 : 0;
    int expect = -1;
    g_log.compare_exchange_strong(expect, v);
    v = g_log.load();
  }
  return v > 0;
}

void log_plan(const Geom& g, const StencilDesc& s, const Choice& c, int64_t nsteps,
              int64_t launches, bool graph) {
  static const char* kinds[] = {"linear", "jacobi5", "diff7", "star9r2", "swe_cgrid", "swe_flux",
                                "source"};
  static const char* dtypes[] = {"f64", "f32", "bf16"};
  static const char* paths[] = {"auto", "tma", "trapezoid", "direct", "march"};
  static const char* bcs[] = {"periodic", "dirichlet", "external"};
  std::vector<int64_t> key{g.ndim, g.n[0], g.n[1], g.n[2], g.dtype, g.nf, s.kind, s.radius,
                           s.stages, c.path, c.tile_x, c.tile_y, c.k, nsteps, graph};
  for (int ax = 0; ax < 3; ++ax) key.insert(key.end(), {g.bc[ax][0], g.bc[ax][1]});
  {
    std::lock_guard<std::mutex> lk(g_log_mu);
    if (!g_logged.insert(key).second) return;
  }
  // extents and boundaries slowest axis first, as the caller's shape
  char ext[64];
  if (g.ndim == 2) std::snprintf(ext, sizeof ext, "%lldx%lld", (long long)g.n[1], (long long)g.n[2]);
  else std::snprintf(ext, sizeof ext, "%lldx%lldx%lld", (long long)g.n[0], (long long)g.n[1],
                     (long long)g.n[2]);
  std::string bc;
  for (int ax = 3 - g.ndim; ax < 3; ++ax) {
    if (ax > 3 - g.ndim) bc += ",";
    bc += bcs[g.bc[ax][0]];
    if (g.bc[ax][1] != g.bc[ax][0]) bc += std::string("/") + bcs[g.bc[ax][1]];
  }
  std::fprintf(stderr,
               "lope: grid %s %s nf=%d bc=[%s] | %s r=%d %s | path=%s tile=%dx%d k=%d | "
               "nsteps=%lld launches=%lld graph=%d\n",
               ext, dtypes[g.dtype], g.nf, bc.c_str(), kinds[s.kind], s.radius,
               s.stages == 1 ? "euler" : s.stages == 2 ? "rk2" : "rk3", paths[c.path], c.tile_x,
               c.tile_y, c.k, (long long)nsteps, (long long)launches, int(graph));
}

// Multi-stage steps as one launch per stage (TMA or direct kernels).  Step j
// starts from b = in (j = 0) or out; with work state W1 (and W2, the second
// state of each work buffer, for RK3):
//   RK2: W1 = E(b); out = 1/2 b + 1/2 E(W1)
//   RK3: W1 = E(b); W2 = 3/4 b + 1/4 E(W1); out = 1/3 b + 2/3 E(W2)
// A combining stage reads b only at the element it writes, so writing out
// while b is out is race-free.
cudaError_t issue_stages(const Geom& g, const StencilDesc& s, const Choice& c,
                         const void* const* in, void* const* out, void* const* work,
                         int64_t nsteps, int* err, cudaStream_t st) {
  const size_t fb = size_t(npts(g)) * esize(g.dtype);
  const int S = s.stages;
  for (int64_t j = 0; j < nsteps; ++j) {
    const void* b[kMaxFields];
    void* w1[kMaxFields];
    void* w2[kMaxFields];
    for (int f = 0; f < g.nf; ++f) {
      b[f] = j == 0 ? in[f] : out[f];
      w1[f] = work[f];
      w2[f] = static_cast<char*>(work[f]) + fb;
    }
    for (int stage = 1; stage <= S; ++stage) {
      StepArgs a = base_args(g, s, err, st);
      a.tile_x = c.tile_x;
      a.tile_y = c.tile_y;
      a.stage = stage;
      if (stage >= 2) rk_coeffs(S, stage, &a.rk_a, &a.rk_b);
      for (int f = 0; f < g.nf; ++f) {
        a.in[f] = stage == 1 ? b[f] : stage == 2 ? w1[f] : w2[f];
        a.out[f] = stage == S ? out[f] : stage == 1 ? w1[f] : w2[f];
        a.base[f] = b[f];
      }
      cudaError_t e;
      if (c.path == kPathTma) e = stage == 1 ? launch_tma(a, nullptr) : launch_tma_stage(a);
      else if (c.path == kPathMarch) e = launch_march(a);
      else e = launch_direct(a, nullptr);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// Issue the launch sequence: ceil(nsteps/k) launches ping-ponging between out
// and work so that the last one writes out.
cudaError_t issue(const Geom& g, const StencilDesc& s, const Choice& c, const void* const* in,
                  void* const* out, void* const* work, int64_t nsteps, int* err, cudaStream_t st) {
  if (s.stages >= 2 && c.path != kPathTrap)
    return issue_stages(g, s, c, in, out, work, nsteps, err, st);
  const int64_t L = (nsteps + c.k - 1) / c.k;
  const void* src[kMaxFields];
  for (int f = 0; f < g.nf; ++f) src[f] = in[f];
  for (int64_t j = 0; j < L; ++j) {
    StepArgs a = base_args(g, s, err, st);
    a.ksteps = int(std::min<int64_t>(c.k, nsteps - j * c.k));
    a.tile_x = c.tile_x;
    a.tile_y = c.tile_y;
    const bool to_out = ((L - 1 - j) & 1) == 0;
    for (int f = 0; f < g.nf; ++f) {
      a.in[f] = src[f];
      a.out[f] = to_out ? out[f] : work[f];
    }
    cudaError_t e;
    switch (c.path) {
      case kPathTma: e = launch_tma(a, nullptr); break;
      case kPathTrap: e = launch_trap2d(a); break;
      case kPathMarch: e = launch_march(a); break;
      default: e = launch_direct(a, nullptr); break;
    }
    if (e != cudaSuccess) return e;
    for (int f = 0; f < g.nf; ++f) src[f] = a.out[f];
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------ graph cache
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
};
using GraphKey = std::vector<int64_t>;
std::mutex g_graph_mu;
std::map<GraphKey, GraphEntry> g_graphs;

GraphKey graph_key(const Geom& g, const StencilDesc& s, const Choice& c, const void* const* in,
                   void* const* out, void* const* work, int64_t nsteps) {
  GraphKey k;
  int dev = 0;
  cudaGetDevice(&dev);
  k.push_back(dev);
  const int64_t* gw = reinterpret_cast<const int64_t*>(&g);
  k.insert(k.end(), gw, gw + sizeof(Geom) / 8);
  const int64_t* sw = reinterpret_cast<const int64_t*>(&s);
  k.insert(k.end(), sw, sw + sizeof(StencilDesc) / 8);
  k.insert(k.end(), {c.path, c.tile_x, c.tile_y, c.k, nsteps});
  for (int f = 0; f < g.nf; ++f) {
    k.push_back(int64_t(reinterpret_cast<uintptr_t>(in[f])));
    k.push_back(int64_t(reinterpret_cast<uintptr_t>(out[f])));
    k.push_back(work ? int64_t(reinterpret_cast<uintptr_t>(work[f])) : 0);
  }
  return k;
}

template <class F>
lope_status run_graph(const GraphKey& key, cudaStream_t st, F&& body) {
  DevState* d = nullptr;
  lope_status rs = dev_state(&d);
  if (rs != LOPE_OK) return rs;
  GraphEntry ent;
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto it = g_graphs.find(key);
    if (it != g_graphs.end()) ent = it->second;
  }
  if (!ent.exec) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(d->capture, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    g_capturing = true;
    g_captured = 0;
    lope_status sb = body(d->capture);
    g_capturing = false;
    e = cudaStreamEndCapture(d->capture, &graph);
    if (sb != LOPE_OK) {
      if (graph) cudaGraphDestroy(graph);
      return sb;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ent.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    ent.kernels = g_captured;
    std::lock_guard<std::mutex> lk(g_graph_mu);
    if (g_graphs.size() > 256) {
      for (auto& kv : g_graphs) cudaGraphExecDestroy(kv.second.exec);
      g_graphs.clear();
    }
    g_graphs[key] = ent;
  }
  cudaError_t e = cudaGraphLaunch(ent.exec, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  count_launches(ent.kernels);
  return LOPE_OK;
}

// The host-only part of an apply: compile a source stencil for the storage
// type, resolve the plan, and check every buffer argument.  A bad call fails
// here, before any CUDA call is made.
lope_status prepare_apply(const lope_grid* grid, const lope_stencil* st, const void* const* in,
                          void* const* out, void* const* work, int64_t nsteps,
                          const lope_launch* cfg, Choice* c, int64_t* L) {
  lope_status rs = check_pair(grid, st);
  if (rs != LOPE_OK) return rs;
  if (nsteps < 0) return fail(LOPE_ERR_INVALID, "nsteps < 0");
  const Geom& g = grid->g;
  const StencilDesc& s = st->s;
  if (st->jit) {  // user source: compile for this storage type first (host only, cached)
    std::string err;
    if ((rs = jit_compile(st->jit, g.dtype, &err)) != LOPE_OK) return fail(rs, err);
  }
  if (has_external(g)) {
    // the caller refreshes an external halo between sweeps (a halo exchange)
    if (nsteps > 1)
      return fail(LOPE_ERR_INVALID, "a grid with an external halo takes one sweep per call");
    if (s.stages != 1)
      return fail(LOPE_ERR_UNSUPPORTED, "multi-stage schemes need a halo exchange per stage");
  }
  if ((rs = resolve(g, s, in, cfg, nullptr, c)) != LOPE_OK) return rs;
  *L = nsteps == 0 ? 0 : (nsteps + c->k - 1) / c->k;
  const bool staged = s.stages >= 2 && c->path != kPathTrap;  // one launch per stage
  if (staged) *L = nsteps * s.stages;
  return check_fields(g, in, out, work, staged ? nsteps >= 1 : *L >= 2, work_states(s), s.radius);
}

lope_status apply_impl(const lope_grid* grid, const lope_stencil* st, const void* const* in,
                       void* const* out, void* const* work, int64_t nsteps, const lope_launch* cfg,
                       cudaStream_t stream) {
  Choice c;
  int64_t L = 0;
  lope_status rs = prepare_apply(grid, st, in, out, work, nsteps, cfg, &c, &L);
  if (rs != LOPE_OK) return rs;
  const Geom& g = grid->g;
  const StencilDesc& s = st->s;
  const int gmode = cfg ? cfg->graph : 0;
  const bool use_graph = gmode == 1 || (gmode == 0 && L >= 8 && npts(g) <= (int64_t(1) << 22));
  if (nsteps > 0 && log_enabled()) log_plan(g, s, c, nsteps, L, use_graph);
  DevState* d = nullptr;
  if ((rs = dev_state(&d)) != LOPE_OK) return rs;
  if (nsteps == 0) {
    for (int f = 0; f < g.nf; ++f) {
      cudaError_t e = cudaMemcpyAsync(out[f], in[f], size_t(npts(g)) * esize(g.dtype),
                                      cudaMemcpyDeviceToDevice, stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    }
    return LOPE_OK;
  }
  if (use_graph) {
    return run_graph(graph_key(g, s, c, in, out, work, nsteps), stream, [&](cudaStream_t cs) {
      cudaError_t e = issue(g, s, c, in, out, work, nsteps, d->err, cs);
      return e == cudaSuccess ? LOPE_OK : cuda_fail(e, "capturing launches");
    });
  }
  cudaError_t e = issue(g, s, c, in, out, work, nsteps, d->err, stream);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return LOPE_OK;
}

// ------------------------------------------------------------------ adjoint
struct AdjLayout {
  int64_t nseg;
  size_t field;  // bytes per state, 256-aligned
  size_t off_ckpt, off_seg, off_tmp, off_lam, off_part, off_scal, total;
  int partials;
};

constexpr int kPartials = 8192;

AdjLayout adj_layout(const Geom& g, int64_t nsteps, int64_t K) {
  AdjLayout L;
  L.nseg = (nsteps + K - 1) / K;
  L.field = (size_t(npts(g)) * esize(g.dtype) + 255) / 256 * 256;
  size_t off = 0;
  L.off_ckpt = off;  // checkpoints 1..nseg-1 and u_T (nseg states)
  off += size_t(L.nseg) * L.field;
  L.off_seg = off;   // recomputed states inside a segment (K-1)
  off += size_t(std::max<int64_t>(K - 1, 0)) * L.field;
  L.off_tmp = off;   // forward work buffer
  off += L.field;
  L.off_lam = off;   // two adjoint buffers
  off += 2 * L.field;
  L.off_part = off;
  L.partials = kPartials;
  off += size_t(kPartials) * sizeof(double);
  L.off_scal = off;  // loss, dL/dc
  off += 256;
  L.total = off;
  return L;
}

lope_status check_linear_for_adjoint(const lope_grid* grid, const lope_stencil* st) {
  lope_status rs = check_pair(grid, st);
  if (rs != LOPE_OK) return rs;
  const StencilDesc& s = st->s;
  if (s.kind == kSwe || s.kind == kSweFlux || s.kind == kUser)
    return fail(LOPE_ERR_UNSUPPORTED, "adjoint needs a single-field linear stencil");
  if (has_external(grid->g))
    return fail(LOPE_ERR_UNSUPPORTED, "adjoint of a grid with an external halo is not implemented");
  if (s.stages != 1) return fail(LOPE_ERR_UNSUPPORTED, "adjoint of a multi-stage scheme is not implemented");
  if (s.kind != kLinear) {
    for (int ax = 0; ax < 3; ++ax)
      for (int sd = 0; sd < 2; ++sd)
        if (grid->g.bc[ax][sd] == kDirichlet && grid->g.bval[ax][sd] != 0.0)
          return fail(LOPE_ERR_UNSUPPORTED, "dL/dc with a non-zero Dirichlet value is not implemented");
  }
  return LOPE_OK;
}

// Forward from u0 to the checkpoints and u_T (u_T written to `uT`).
lope_status forward_ckpt_impl(const lope_grid* grid, const lope_stencil* st, const void* u0,
                              void* uT, int64_t nsteps, int64_t K, char* ws, const AdjLayout& L,
                              cudaStream_t stream) {
  void* tmp = ws + L.off_tmp;
  const void* cur = u0;
  for (int64_t i = 0; i < L.nseg; ++i) {
    const int64_t len = std::min<int64_t>(K, nsteps - i * K);
    void* dst = (i == L.nseg - 1) ? uT : static_cast<void*>(ws + L.off_ckpt + size_t(i) * L.field);
    const void* in1[1] = {cur};
    void* out1[1] = {dst};
    void* work1[1] = {tmp};
    lope_launch cfg = {0, 0, 0, 0, -1};
    lope_status rs = apply_impl(grid, st, in1, out1, work1, len, &cfg, stream);
    if (rs != LOPE_OK) return rs;
    cur = dst;
  }
  return LOPE_OK;
}

StencilDesc reflected(const StencilDesc& s) {
  StencilDesc r = s;
  const int R = s.radius, side = 2 * R + 1;
  for (int ax = 0; ax < 3; ++ax)
    for (int d = 0; d < side; ++d) r.star_w[ax][d] = s.star_w[ax][side - 1 - d];
  const int cnt = (s.ndim == 3 ? side : 1) * side * side;
  for (int i = 0; i < cnt; ++i) r.box[i] = s.box[cnt - 1 - i];
  return r;
}

// Reverse sweep: lambda from `lamT` back to grad_u0, recomputing states from
// checkpoints; dL/dc accumulated into per-block partials, finalised into gc.
lope_status reverse_impl(const lope_grid* grid, const lope_stencil* st, const void* u0,
                         const void* lamT, int64_t nsteps, int64_t K, void* grad_u0, double* gc,
                         char* ws, const AdjLayout& L, int* err, cudaStream_t stream) {
  const Geom& g = grid->g;
  Geom ga = g;  // lambda's halo: Dirichlet sides read zero
  for (int ax = 0; ax < 3; ++ax)
    for (int sd = 0; sd < 2; ++sd) ga.bval[ax][sd] = 0.0;
  const StencilDesc& s = st->s;
  const bool diffusion = s.kind != kLinear;
  const StencilDesc sa = diffusion ? s : reflected(s);
  double* partials = reinterpret_cast<double*>(ws + L.off_part);
  cudaError_t e = cudaMemsetAsync(partials, 0, sizeof(double) * L.partials, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  StepArgs probe = base_args(ga, sa, err, stream);
  probe.in[0] = lamT;
  probe.adjoint = diffusion;
  const bool tma = tma_supported(probe);
  int blocks_used = 0;
  const void* lam = lamT;
  int64_t m = 0;  // adjoint steps done
  for (int64_t i = L.nseg - 1; i >= 0; --i) {
    const int64_t s0 = i * K, len = std::min<int64_t>(K, nsteps - s0);
    const void* ck = i == 0 ? u0 : static_cast<const void*>(ws + L.off_ckpt + size_t(i - 1) * L.field);
    // recompute u_{s0+1} .. u_{s0+len-1}
    const void* prev = ck;
    for (int64_t j = 1; j < len; ++j) {
      void* dst = ws + L.off_seg + size_t(j - 1) * L.field;
      const void* in1[1] = {prev};
      void* out1[1] = {dst};
      lope_launch cfg = {0, 0, 0, 0, -1};
      lope_status rs = apply_impl(grid, st, in1, out1, nullptr, 1, &cfg, stream);
      if (rs != LOPE_OK) return rs;
      prev = dst;
    }
    for (int64_t j = len - 1; j >= 0; --j, ++m) {
      const void* ut = j == 0 ? ck : static_cast<const void*>(ws + L.off_seg + size_t(j - 1) * L.field);
      void* dst = (m == nsteps - 1) ? grad_u0
                                    : static_cast<void*>(ws + L.off_lam + size_t(m & 1) * L.field);
      StepArgs a = base_args(ga, sa, err, stream);
      a.in[0] = lam;
      a.out[0] = dst;
      a.adjoint = diffusion;
      a.ut = ut;
      a.partials = partials;
      a.partial_count = L.partials;
      int b = 0;
      e = tma ? launch_tma(a, &b) : launch_direct(a, &b);
      if (e != cudaSuccess) return cuda_fail(e, "adjoint kernel launch");
      blocks_used = std::max(blocks_used, b);
      lam = dst;
    }
  }
  if (gc) {
    if (diffusion) {
      e = launch_finalize(partials, std::max(blocks_used, 1), gc, 0, stream);
    } else {
      e = cudaMemsetAsync(gc, 0, sizeof(double), stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "finalize dL/dc");
  }
  return LOPE_OK;
}

// Key of a captured adjoint sequence: everything that the launches depend on.
GraphKey adjoint_key(int kind, const lope_grid* grid, const lope_stencil* st,
                     std::initializer_list<const void*> ptrs, int64_t nsteps, int64_t K) {
  GraphKey k;
  int dev = 0;
  cudaGetDevice(&dev);
  k.push_back(-1000 - kind);
  k.push_back(dev);
  const int64_t* gw = reinterpret_cast<const int64_t*>(&grid->g);
  k.insert(k.end(), gw, gw + sizeof(Geom) / 8);
  const int64_t* sw = reinterpret_cast<const int64_t*>(&st->s);
  k.insert(k.end(), sw, sw + sizeof(StencilDesc) / 8);
  for (const void* p : ptrs) k.push_back(int64_t(reinterpret_cast<uintptr_t>(p)));
  k.push_back(nsteps);
  k.push_back(K);
  return k;
}

// ------------------------------------------------------------------ batch
struct BatchPlan {
  std::vector<BatchGrid> host;
  BatchGrid* pinned = nullptr;
  BatchPlanDev dev;
  cudaGraphExec_t exec = nullptr;
  int blocks = 0;
  int64_t kernels = 1;  // kernel launches per replay
  ~BatchPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (pinned) cudaFreeHost(pinned);
  }
};
std::mutex g_batch_mu;
std::map<std::vector<int64_t>, std::shared_ptr<BatchPlan>> g_batch;

// Batch workspace: the barrier and claim counters (256 B), the grid list, and
// one record per tile of the two-sweep batched tiles (64 x 64 tiles).
size_t round256(size_t b) { return (b + 255) / 256 * 256; }
int64_t batch_tb2_items(int n, const lope_grid* const* grids) {
  int64_t items = 0;
  for (int i = 0; i < n; ++i)
    items += ((grids[i]->g.n[2] + kBatchTb2X - 1) / kBatchTb2X) *
             ((grids[i]->g.n[1] + kBatchTb2Y - 1) / kBatchTb2Y);
  return items;
}
size_t batch_ws_bytes(int n, const lope_grid* const* grids) {
  return 256 + round256(size_t(n) * sizeof(BatchGrid)) +
         round256(size_t(batch_tb2_items(n, grids)) * sizeof(BatchItem));
}

// Batch autotuner cache: the fastest (tile, depth) per batch signature (grid
// shapes and boundaries, dtype, stencil), filled by lope_autotune_batch.
using BatchSig = std::vector<int64_t>;
std::mutex g_btune_mu;
std::map<BatchSig, Choice> g_btune;

BatchSig batch_sig(int n, const lope_grid* const* grids, const StencilDesc& s) {
  BatchSig k = {int64_t(n), int64_t(grids[0]->g.dtype), s.kind, s.radius, s.stages,
                int64_t(reinterpret_cast<uintptr_t>(s.jit))};
  for (int i = 0; i < 4; ++i) {
    int64_t b;
    std::memcpy(&b, &s.prm[i], 8);
    k.push_back(b);
  }
  for (int i = 0; i < n; ++i) {
    const Geom& g = grids[i]->g;
    k.push_back(g.n[1]);
    k.push_back(g.n[2]);
    for (int ax = 1; ax < 3; ++ax)
      for (int sd = 0; sd < 2; ++sd) {
        k.push_back(g.bc[ax][sd]);
        int64_t b;
        std::memcpy(&b, &g.bval[ax][sd], 8);
        k.push_back(b);
      }
  }
  return k;
}

// ------------------------------------------------------------------ tune cache file
// The autotuners' choices as a text file, one entry per line:
//   lope-tune 1 <gpu> grid <ndim> <n0> <n1> <n2> <dtype> <kind> <radius> <star> <bcs> <nf> <stages> : <path> <tile_x> <tile_y> <k>
//   lope-tune 1 <gpu> batch <m> <m signature integers> : <path> <tile_x> <tile_y> <k>
// <gpu> is the device name with blanks replaced by '_'.  Entries of source
// stencils are not written (their keys hold a process-local pointer).
std::string gpu_tag(const char* name) {
  std::string t(name);
  for (char& ch : t)
    if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
  return t;
}

lope_status gpu_tag_of(const char* gpu_name, std::string* out) {
  if (gpu_name) {
    *out = gpu_tag(gpu_name);
  } else {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess)
      return cuda_fail(e, "cudaGetDeviceProperties");
    *out = gpu_tag(prop.name);
  }
  if (out->empty()) return fail(LOPE_ERR_INVALID, "empty GPU name");
  return LOPE_OK;
}

bool choice_in_range(const Choice& c) {
  return c.path >= kPathTma && c.path <= kPathMarch && c.tile_x >= 0 && c.tile_x <= 256 &&
         c.tile_y >= 0 && c.tile_y <= 256 && c.k >= 1 && c.k <= 8;
}

// One line of a cache file; false if it is malformed or names another GPU.
bool parse_tune_line(const std::string& line, const std::string& gpu, bool* batch, TuneKey* gk,
                     BatchSig* bk, Choice* c) {
  std::istringstream is(line);
  std::string magic, tag, kind, colon;
  int version = 0;
  if (!(is >> magic >> version >> tag >> kind) || magic != "lope-tune" || version != 1 || tag != gpu)
    return false;
  if (kind == "grid") {
    long long v[11];
    for (auto& x : v)
      if (!(is >> x)) return false;
    if (v[0] < 2 || v[0] > 3 || v[1] < 1 || v[2] < 1 || v[3] < 1 || v[4] < 0 || v[4] > 2) return false;
    *gk = TuneKey(int(v[0]), v[1], v[2], v[3], int(v[4]), int(v[5]), int(v[6]), int(v[7]), int(v[8]),
                  int(v[9]), int(v[10]), 0);
    *batch = false;
  } else if (kind == "batch") {
    long long m = 0;
    if (!(is >> m) || m < 6 || m > (1 << 22)) return false;
    bk->assign(size_t(m), 0);
    for (auto& x : *bk) {
      long long y;
      if (!(is >> y)) return false;
      x = y;
    }
    if ((*bk)[5] != 0) return false;
    *batch = true;
  } else {
    return false;
  }
  if (!(is >> colon >> c->path >> c->tile_x >> c->tile_y >> c->k) || colon != ":") return false;
  if (!choice_in_range(*c)) return false;
  if (*batch && !((c->path == kPathTrap && c->tile_x >= 8 && c->tile_y >= 1) ||
                  (c->path == kPathTma && c->tile_x == kBatchTb2X && c->tile_y == kBatchTb2Y &&
                   c->k == 2)))
    return false;
  return true;
}

}  // namespace

void count_launches(int64_t n) {
  if (g_capturing) g_captured += n;
  else g_launches.fetch_add(n);
}

}  // namespace lope

using namespace lope;

lope_status lope_fail_external(lope_status st, const char* msg) { return fail(st, msg); }

// ====================================================================== C ABI
extern "C" {

const char* lope_last_error(void) { return g_last_error.c_str(); }
const char* lope_version(void) { return "lope-gb300 0.1 (sm_103a)"; }
int64_t lope_launch_count(void) { return g_launches.load(); }

lope_status lope_grid_create(lope_grid** grid, int ndim, const int64_t* extents, const int* halo_lo,
                             const int* halo_hi, lope_dtype storage, int nfields) {
  if (!grid || !extents || !halo_lo || !halo_hi) return fail(LOPE_ERR_INVALID, "NULL argument");
  if (ndim != 2 && ndim != 3) return fail(LOPE_ERR_INVALID, "ndim must be 2 or 3");
  if (storage != LOPE_F64 && storage != LOPE_F32 && storage != LOPE_BF16)
    return fail(LOPE_ERR_INVALID, "unknown dtype");
  if (nfields < 1 || nfields > kMaxFields) return fail(LOPE_ERR_INVALID, "nfields must be 1..3");
  auto* h = new (std::nothrow) lope_grid;
  if (!h) return fail(LOPE_ERR_ALLOC, "out of host memory");
  std::memset(h, 0, sizeof(*h));
  h->g.ndim = ndim;
  h->g.dtype = storage;
  h->g.nf = nfields;
  const int off = 3 - ndim;
  for (int ax = 0; ax < 3; ++ax) h->g.n[ax] = 1;
  for (int i = 0; i < ndim; ++i) {
    if (extents[i] < 1 || extents[i] > (int64_t(1) << 31) || halo_lo[i] < 0 || halo_hi[i] < 0 ||
        halo_lo[i] > 4 || halo_hi[i] > 4) {
      delete h;
      return fail(LOPE_ERR_INVALID, "extent or halo out of range");
    }
    h->g.n[off + i] = extents[i];
    h->halo_lo[off + i] = halo_lo[i];
    h->halo_hi[off + i] = halo_hi[i];
  }
  if (h->g.n[0] * h->g.n[1] * h->g.n[2] > (int64_t(1) << 34)) {
    delete h;
    return fail(LOPE_ERR_INVALID, "grid too large");
  }
  *grid = h;
  return LOPE_OK;
}

void lope_grid_destroy(lope_grid* grid) { delete grid; }

lope_status lope_set_boundary(lope_grid* grid, int axis, int side, lope_bc kind, double value) {
  if (!grid) return fail(LOPE_ERR_INVALID, "NULL grid");
  const int nd = grid->g.ndim;
  if (axis < -1 || axis >= nd || side < -1 || side > 1) return fail(LOPE_ERR_INVALID, "bad axis or side");
  if (kind != LOPE_BC_PERIODIC && kind != LOPE_BC_DIRICHLET && kind != LOPE_BC_EXTERNAL)
    return fail(LOPE_ERR_INVALID, "bad boundary kind");
  if (kind == LOPE_BC_PERIODIC && side != -1) return fail(LOPE_ERR_INVALID, "periodic applies to both sides");
  if (kind == LOPE_BC_EXTERNAL && axis != 0)
    return fail(LOPE_ERR_INVALID, "an external halo belongs to the slowest axis (axis 0)");
  if (!std::isfinite(value)) return fail(LOPE_ERR_INVALID, "non-finite Dirichlet value");
  const int off = 3 - nd;
  for (int a = 0; a < nd; ++a) {
    if (axis != -1 && a != axis) continue;
    for (int sd = 0; sd < 2; ++sd) {
      if (side != -1 && sd != side) continue;
      grid->g.bc[off + a][sd] = kind == LOPE_BC_PERIODIC ? kPeriodic
                                : kind == LOPE_BC_EXTERNAL ? kExternal : kDirichlet;
      grid->g.bval[off + a][sd] = kind == LOPE_BC_DIRICHLET ? value : 0.0;
    }
    // an axis cannot be periodic on one side only: the other side becomes
    // Dirichlet 0
    for (int sd = 0; sd < 2; ++sd)
      if (grid->g.bc[off + a][sd] == kPeriodic && grid->g.bc[off + a][1 - sd] != kPeriodic) {
        grid->g.bc[off + a][sd] = kDirichlet;
        grid->g.bval[off + a][sd] = 0.0;
      }
  }
  return LOPE_OK;
}

lope_status lope_stencil_create_builtin(lope_stencil** stencil, const char* name,
                                        const double* params, int nparams) {
  if (!stencil || !name) return fail(LOPE_ERR_INVALID, "NULL argument");
  auto* h = new (std::nothrow) lope_stencil;
  if (!h) return fail(LOPE_ERR_ALLOC, "out of host memory");
  std::memset(h, 0, sizeof(*h));
  StencilDesc& s = h->s;
  s.star = true;
  s.stages = 1;
  std::string n(name);
  int want = 1;
  if (n == "jacobi5") { s.kind = kJacobi5; s.ndim = 2; s.radius = 1; }
  else if (n == "diff7") { s.kind = kDiff7; s.ndim = 3; s.radius = 1; }
  else if (n == "star9r2") { s.kind = kStar9r2; s.ndim = 2; s.radius = 2; }
  else if (n == "swe_cgrid") { s.kind = kSwe; s.ndim = 2; s.radius = 1; want = 3; }
  else if (n == "swe_flux") { s.kind = kSweFlux; s.ndim = 2; s.radius = 1; s.star = false; want = 4; }
  else { delete h; return fail(LOPE_ERR_INVALID, "unknown builtin stencil name"); }
  if (nparams != want || !params) { delete h; return fail(LOPE_ERR_INVALID, "wrong parameter count"); }
  for (int i = 0; i < want; ++i) {
    if (!std::isfinite(params[i])) { delete h; return fail(LOPE_ERR_INVALID, "non-finite parameter"); }
    s.prm[i] = params[i];
  }
  h->nf = stencil_nf(s);
  *stencil = h;
  return LOPE_OK;
}

lope_status lope_stencil_create_linear(lope_stencil** stencil, int ndim, int radius,
                                       const double* weights) {
  if (!stencil || !weights) return fail(LOPE_ERR_INVALID, "NULL argument");
  if ((ndim != 2 && ndim != 3) || radius < 1 || radius > kMaxRadius)
    return fail(LOPE_ERR_INVALID, "ndim must be 2/3 and radius 1..2");
  auto* h = new (std::nothrow) lope_stencil;
  if (!h) return fail(LOPE_ERR_ALLOC, "out of host memory");
  std::memset(h, 0, sizeof(*h));
  StencilDesc& s = h->s;
  s.kind = kLinear;
  s.ndim = ndim;
  s.radius = radius;
  s.stages = 1;
  const int side = 2 * radius + 1, zs = ndim == 3 ? side : 1, zr = ndim == 3 ? radius : 0;
  bool star = true;
  for (int dz = 0; dz < zs; ++dz)
    for (int dy = 0; dy < side; ++dy)
      for (int dx = 0; dx < side; ++dx) {
        const double w = weights[(dz * side + dy) * side + dx];
        if (!std::isfinite(w)) { delete h; return fail(LOPE_ERR_INVALID, "non-finite weight"); }
        s.box[(dz * side + dy) * side + dx] = w;
        const int ox = dx - radius, oy = dy - radius, oz = dz - zr;
        const int nz = (ox != 0) + (oy != 0) + (oz != 0);
        if (nz > 1 && w != 0.0) star = false;
        if (nz == 0) s.star_w[0][radius] = w;
        else if (ox != 0 && nz == 1) s.star_w[0][ox + radius] = w;
        else if (oy != 0 && nz == 1) s.star_w[1][oy + radius] = w;
        else if (oz != 0 && nz == 1) s.star_w[2][oz + radius] = w;
      }
  s.star = star;
  h->nf = 1;
  *stencil = h;
  return LOPE_OK;
}

void lope_stencil_destroy(lope_stencil* stencil) {
  if (!stencil) return;
  if (stencil->jit) lope::jit_destroy(stencil->jit);
  delete stencil;
}

// The taps U(f, dx, dy[, dz]) of a local-function body whose arguments are all
// integer literals must lie inside the declared halo (Sec. 3.5: no
// out-of-bounds indexing), read an existing field and, for a function
// declared star-shaped, lie on an axis.  Taps with computed arguments are
// checked on the device when they run.  Returns an empty string or the reason.
std::string check_literal_taps(const std::string& text, int ndim, int radius, int nf, bool star) {
  auto ident = [](char c) { return std::isalnum(static_cast<unsigned char>(c)) || c == '_'; };
  std::string body;  // the text without comments
  for (size_t i = 0; i < text.size(); ++i) {
    if (text.compare(i, 2, "//") == 0) {
      while (i < text.size() && text[i] != '\n') ++i;
    } else if (text.compare(i, 2, "/*") == 0) {
      const size_t e = text.find("*/", i + 2);
      i = e == std::string::npos ? text.size() : e + 1;
      body += ' ';
      continue;
    }
    if (i < text.size()) body += text[i];
  }
  for (size_t i = 0; (i = body.find('U', i)) != std::string::npos; ++i) {
    if (i > 0 && ident(body[i - 1])) continue;
    size_t j = i + 1;
    while (j < body.size() && std::isspace(static_cast<unsigned char>(body[j]))) ++j;
    if (j >= body.size() || body[j] != '(') continue;
    // the argument list up to the matching parenthesis, split at top-level commas
    std::vector<std::string> args(1);
    int depth = 0;
    size_t k = j + 1;
    for (; k < body.size(); ++k) {
      const char c = body[k];
      if (c == '(') ++depth;
      if (c == ')' && depth-- == 0) break;
      if (c == ',' && depth == 0) args.emplace_back();
      else args.back() += c;
    }
    std::vector<long> v;
    for (auto& a : args) {
      std::string t;
      for (char c : a)
        if (!std::isspace(static_cast<unsigned char>(c))) t += c;
      size_t q = (!t.empty() && (t[0] == '-' || t[0] == '+')) ? 1 : 0;
      if (q >= t.size() || t.find_first_not_of("0123456789", q) != std::string::npos) {
        v.clear();
        break;
      }
      v.push_back(std::strtol(t.c_str(), nullptr, 10));
    }
    if (v.empty()) continue;  // computed arguments: checked when the kernel runs
    const std::string tap = body.substr(i, k + 1 - i);
    if (int(v.size()) != ndim + 1 && !(ndim == 3 && v.size() == 3))
      return "tap " + tap + " has the wrong number of arguments";
    if (v[0] < 0 || v[0] >= nf) return "tap " + tap + " reads a field the function does not have";
    int nonzero = 0;
    for (size_t a = 1; a < v.size(); ++a) {
      if (v[a] < -radius || v[a] > radius)
        return "tap " + tap + " reads beyond the declared halo of radius " + std::to_string(radius) +
               " (Sec. 3.5: no out-of-bounds indexing)";
      nonzero += v[a] != 0;
    }
    if (star && nonzero > 1)
      return "tap " + tap + " reads a corner of a function declared star-shaped (box = 0)";
  }
  return "";
}

lope_status lope_stencil_create_source(lope_stencil** stencil, int ndim, int radius, int nfields,
                                       int box, const char* body, const double* params,
                                       int nparams) {
  if (!stencil || !body) return fail(LOPE_ERR_INVALID, "NULL argument");
  if ((ndim != 2 && ndim != 3) || radius < 1 || radius > kMaxRadius)
    return fail(LOPE_ERR_INVALID, "ndim must be 2/3 and radius 1..2");
  if (nfields < 1 || nfields > kMaxFields) return fail(LOPE_ERR_INVALID, "nfields must be 1..3");
  if (nparams < 0 || nparams > kUserParams || (nparams > 0 && !params))
    return fail(LOPE_ERR_INVALID, "at most 8 parameters");
  for (int i = 0; i < nparams; ++i)
    if (!std::isfinite(params[i])) return fail(LOPE_ERR_INVALID, "non-finite parameter");
  const std::string bad = check_literal_taps(body, ndim, radius, nfields, box == 0);
  if (!bad.empty()) return fail(LOPE_ERR_INVALID, bad);
  auto* h = new (std::nothrow) lope_stencil;
  if (!h) return fail(LOPE_ERR_ALLOC, "out of host memory");
  std::memset(h, 0, sizeof(*h));
  StencilDesc& s = h->s;
  s.kind = kUser;
  s.ndim = ndim;
  s.radius = radius;
  s.stages = 1;
  s.star = box == 0;
  s.user_nf = nfields;
  for (int i = 0; i < nparams && i < 4; ++i) s.prm[i] = params[i];
  lope_status rs = jit_create(body, ndim, radius, nfields, s.star, params, nparams, &h->jit);
  if (rs != LOPE_OK) {
    delete h;
    return fail(rs, "out of host memory");
  }
  s.jit = h->jit;
  h->nf = nfields;
  *stencil = h;
  return LOPE_OK;
}

lope_status lope_stencil_compile(const lope_stencil* stencil, lope_dtype storage) {
  if (!stencil) return fail(LOPE_ERR_INVALID, "NULL stencil");
  if (storage != LOPE_F64 && storage != LOPE_F32 && storage != LOPE_BF16)
    return fail(LOPE_ERR_INVALID, "unknown dtype");
  if (!stencil->jit) return LOPE_OK;  // builtin and linear stencils are compiled with the library
  std::string err;
  lope_status rs = jit_compile(stencil->jit, int(storage), &err);
  if (rs != LOPE_OK) return fail(rs, err);
  return LOPE_OK;
}

lope_status lope_stencil_set_scheme(lope_stencil* stencil, lope_scheme scheme) {
  if (!stencil) return fail(LOPE_ERR_INVALID, "NULL stencil");
  if (scheme != LOPE_SCHEME_EULER && scheme != LOPE_SCHEME_RK2 && scheme != LOPE_SCHEME_RK3)
    return fail(LOPE_ERR_INVALID, "unknown time-stepping scheme");
  stencil->s.stages = int(scheme);
  return LOPE_OK;
}

lope_status lope_work_states(const lope_stencil* stencil, int* states) {
  if (!stencil || !states) return fail(LOPE_ERR_INVALID, "NULL argument");
  *states = work_states(stencil->s);
  return LOPE_OK;
}

lope_status lope_apply(const lope_grid* grid, const lope_stencil* stencil, const void* const* in,
                       void* const* out, void* const* work, int64_t nsteps, void* cuda_stream) {
  return apply_impl(grid, stencil, in, out, work, nsteps, nullptr,
                    static_cast<cudaStream_t>(cuda_stream));
}

lope_status lope_apply_with(const lope_grid* grid, const lope_stencil* stencil,
                            const void* const* in, void* const* out, void* const* work,
                            int64_t nsteps, const lope_launch* cfg, void* cuda_stream) {
  return apply_impl(grid, stencil, in, out, work, nsteps, cfg,
                    static_cast<cudaStream_t>(cuda_stream));
}

lope_status lope_plan(const lope_grid* grid, const lope_stencil* stencil, const void* const* in,
                      void* const* out, void* const* work, int64_t nsteps, const lope_launch* cfg,
                      lope_launch* plan, int64_t* launches) {
  if (!plan) return fail(LOPE_ERR_INVALID, "NULL plan");
  Choice c;
  int64_t L = 0;
  lope_status rs = prepare_apply(grid, stencil, in, out, work, nsteps, cfg, &c, &L);
  if (rs != LOPE_OK) return rs;
  const int gmode = cfg ? cfg->graph : 0;
  const bool use_graph = gmode == 1 || (gmode == 0 && L >= 8 && npts(grid->g) <= (int64_t(1) << 22));
  plan->path = c.path;
  plan->tile_x = c.tile_x;
  plan->tile_y = c.tile_y;
  plan->tsteps = c.k;
  plan->graph = use_graph ? 1 : -1;
  if (launches) *launches = L;
  return LOPE_OK;
}

lope_status lope_apply_host(const lope_grid* grid, const lope_stencil* stencil,
                            const void* const* host_in, void* const* host_out,
                            void* const* dev_in, void* const* dev_out, void* const* dev_work,
                            int64_t nsteps, void* cuda_stream) {
  lope_status rs = check_pair(grid, stencil);
  if (rs != LOPE_OK) return rs;
  if (!host_in || !host_out || !dev_in) return fail(LOPE_ERR_INVALID, "NULL field array");
  const Geom& g = grid->g;
  // every argument, host pointers included, is checked before the first copy is issued
  for (int f = 0; f < g.nf; ++f)
    if (!host_in[f] || !host_out[f]) return fail(LOPE_ERR_INVALID, "NULL host field pointer");
  {
    Choice c;
    int64_t L = 0;
    if ((rs = prepare_apply(grid, stencil, dev_in, dev_out, dev_work, nsteps, nullptr, &c, &L)) !=
        LOPE_OK)
      return rs;
  }
  const size_t bytes = size_t(npts(g)) * esize(g.dtype);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  for (int f = 0; f < g.nf; ++f) {
    cudaError_t e = cudaMemcpyAsync(dev_in[f], host_in[f], bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (host to device)");
  }
  if ((rs = apply_impl(grid, stencil, dev_in, dev_out, dev_work, nsteps, nullptr, st)) != LOPE_OK)
    return rs;
  for (int f = 0; f < g.nf; ++f) {
    cudaError_t e = cudaMemcpyAsync(host_out[f], dev_out[f], bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (device to host)");
  }
  return LOPE_OK;
}

lope_status lope_autotune(const lope_grid* grid, const lope_stencil* stencil,
                          const void* const* in, void* const* out, void* const* work,
                          int64_t nsteps, lope_launch* best, double* best_ms, void* cuda_stream) {
  lope_status rs = check_pair(grid, stencil);
  if (rs != LOPE_OK) return rs;
  if (nsteps < 1) return fail(LOPE_ERR_INVALID, "autotune needs nsteps >= 1");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const Geom& g = grid->g;
  std::vector<lope_launch> cands;
  cands.push_back({kPathTma, 0, 0, 1, -1});
  if (g.ndim == 2) {
    const int tiles[][2] = {{64, 32}, {128, 16}, {64, 16}, {32, 32}, {128, 32}};
    for (auto& t : tiles)
      for (int k : {1, 2, 3, 4, 6, 8}) cands.push_back({kPathTrap, t[0], t[1], k, -1});
  }
  if (g.ndim == 3) cands.push_back({kPathMarch, 0, 0, 1, -1});
  cands.push_back({kPathDirect, 0, 0, 1, -1});
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double bms = 1e300;
  lope_launch bl = {0, 0, 0, 0, 0};
  for (const auto& c : cands) {
    if (apply_impl(grid, stencil, in, out, work, nsteps, &c, st) != LOPE_OK) continue;  // warm-up / support check
    cudaEventRecord(e0, st);
    rs = apply_impl(grid, stencil, in, out, work, nsteps, &c, st);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || rs != LOPE_OK) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < bms) {
      bms = ms;
      bl = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g_last_error = "no error";
  if (bl.path == 0) return fail(LOPE_ERR_UNSUPPORTED, "no launch path supports this grid/stencil");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(g, stencil->s)] = {bl.path, bl.tile_x, bl.tile_y, bl.tsteps > 0 ? bl.tsteps : 1};
  }
  if (best) *best = bl;
  if (best_ms) *best_ms = bms;
  return LOPE_OK;
}

lope_status lope_batch_workspace_size(int n, const lope_grid* const* grids,
                                      const lope_stencil* stencil, const lope_launch* cfg,
                                      size_t* bytes) {
  (void)cfg;
  if (n < 1 || !grids || !stencil || !bytes) return fail(LOPE_ERR_INVALID, "bad argument");
  for (int i = 0; i < n; ++i)
    if (!grids[i]) return fail(LOPE_ERR_INVALID, "NULL grid");
  *bytes = batch_ws_bytes(n, grids);
  return LOPE_OK;
}

lope_status lope_apply_batch(int n, const lope_grid* const* grids, const lope_stencil* stencil,
                             const void* const* in, void* const* out, void* const* work,
                             int64_t nsteps, const lope_launch* cfg, void* workspace,
                             size_t workspace_bytes, void* cuda_stream) {
  if (n < 1 || !grids || !stencil || !in || !out || !workspace)
    return fail(LOPE_ERR_INVALID, "NULL argument");
  if (nsteps < 1) return fail(LOPE_ERR_INVALID, "nsteps must be >= 1");
  for (int i = 0; i < n; ++i)
    if (!grids[i]) return fail(LOPE_ERR_INVALID, "NULL grid");
  if (workspace_bytes < batch_ws_bytes(n, grids))
    return fail(LOPE_ERR_ALLOC, "batch workspace too small");
  if (!aligned16(workspace)) return fail(LOPE_ERR_INVALID, "workspace not 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const StencilDesc& s = stencil->s;
  if (s.stages != 1) return fail(LOPE_ERR_UNSUPPORTED, "the batched kernel runs forward-Euler stencils only");
  const int dtype = grids[0]->g.dtype;
  for (int i = 0; i < n; ++i) {
    lope_status rs = check_pair(grids[i], stencil);
    if (rs != LOPE_OK) return rs;
    if (grids[i]->g.ndim != 2 || grids[i]->g.nf != 1 || grids[i]->g.dtype != dtype)
      return fail(LOPE_ERR_INVALID, "batch grids must be 2D, single-field, same dtype");
    if (has_external(grids[i]->g))
      return fail(LOPE_ERR_UNSUPPORTED, "batched grids take periodic or Dirichlet boundaries");
    const void* in1[1] = {in[i]};
    void* out1[1] = {out[i]};
    void* work1[1] = {work ? work[i] : nullptr};
    if ((rs = check_fields(grids[i]->g, in1, out1, work1, true)) != LOPE_OK) return rs;
  }
  // The two-sweep register tiles (path 1: 64 x 64 tiles, two sweeps per
  // pass) serve FP32 star functions of radius 1-2 (jacobi5, star9r2, linear
  // star tables) and are the default there; other batches take the trapezoid
  // tiles (path 2, 64 x 32, four sweeps per pass).  A choice remembered by the
  // batch autotuner comes first; cfg overrides either.
  const bool tb2_ok = dtype == kF32 && s.star && s.radius <= 2 &&
                      (s.kind == kJacobi5 || s.kind == kStar9r2 || s.kind == kLinear);
  Choice tuned = tb2_ok ? Choice{kPathTma, kBatchTb2X, kBatchTb2Y, 2} : Choice{kPathTrap, 64, 32, 4};
  if (!cfg || cfg->path == kPathAuto || cfg->tile_x <= 0 || cfg->tile_y <= 0 || cfg->tsteps <= 0) {
    std::lock_guard<std::mutex> lk(g_btune_mu);
    auto it = g_btune.find(batch_sig(n, grids, s));
    if (it != g_btune.end()) tuned = it->second;
  }
  const int path = cfg && cfg->path != kPathAuto ? cfg->path : tuned.path;
  if (path != kPathTma && path != kPathTrap)
    return fail(LOPE_ERR_UNSUPPORTED, "the batched launch runs trapezoid (2) or two-sweep (1) tiles");
  const int mode = path == kPathTma ? 1 : 0;
  const int tx = mode ? kBatchTb2X : cfg && cfg->tile_x > 0 ? cfg->tile_x : tuned.tile_x;
  const int ty = mode ? kBatchTb2Y : cfg && cfg->tile_y > 0 ? cfg->tile_y : tuned.tile_y;
  const int k = mode ? 2 : cfg && cfg->tsteps > 0 ? cfg->tsteps : tuned.k;
  if (tx < 8 || tx > 256 || ty < 1 || ty > 256 || k < 1 || k > 8)
    return fail(LOPE_ERR_INVALID, "bad batch tile or depth");
  if (mode && cfg && cfg->tsteps > 0 && cfg->tsteps != 2)
    return fail(LOPE_ERR_UNSUPPORTED, "the two-sweep batched tiles run two sweeps per pass");
  DevState* d = nullptr;
  lope_status rs = dev_state(&d);
  if (rs != LOPE_OK) return rs;
  const int maxb = batch_max_blocks(s, dtype, tx, ty, k, mode);
  if (maxb <= 0) return fail(LOPE_ERR_UNSUPPORTED, "batched kernel does not support this stencil/tile");

  const int64_t wait_ms = g_wait_limit_ms.load(), skip = g_skip_arrive.load();
  std::vector<int64_t> key = {int64_t(n), int64_t(dtype), s.kind, tx, ty, k, nsteps,
                              int64_t(reinterpret_cast<uintptr_t>(workspace)), wait_ms, skip, mode};
  const int64_t* sw = reinterpret_cast<const int64_t*>(&s);
  key.insert(key.end(), sw, sw + sizeof(StencilDesc) / 8);
  for (int i = 0; i < n; ++i) {
    const Geom& g = grids[i]->g;
    key.insert(key.end(), {g.n[1], g.n[2], int64_t(reinterpret_cast<uintptr_t>(in[i])),
                           int64_t(reinterpret_cast<uintptr_t>(out[i])),
                           int64_t(reinterpret_cast<uintptr_t>(work[i]))});
    for (int ax = 1; ax < 3; ++ax)
      for (int sd = 0; sd < 2; ++sd) {
        key.push_back(g.bc[ax][sd]);
        int64_t b;
        std::memcpy(&b, &g.bval[ax][sd], 8);
        key.push_back(b);
      }
  }
  std::shared_ptr<BatchPlan> plan;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto it = g_batch.find(key);
    if (it != g_batch.end()) plan = it->second;
  }
  if (!plan) {
    plan = std::make_shared<BatchPlan>();
    int items = 0;
    plan->host.resize(n);
    for (int i = 0; i < n; ++i) {
      const Geom& g = grids[i]->g;
      BatchGrid& b = plan->host[i];
      b.in = in[i];
      b.out = out[i];
      b.work = work[i];
      b.nx = int(g.n[2]);
      b.ny = int(g.n[1]);
      for (int sd = 0; sd < 2; ++sd) {
        b.bc[0][sd] = g.bc[1][sd];
        b.bval[0][sd] = g.bval[1][sd];
        b.bc[1][sd] = g.bc[2][sd];
        b.bval[1][sd] = g.bval[2][sd];
      }
      b.tiles_x = (b.nx + tx - 1) / tx;
      b.first_item = items;
      items += b.tiles_x * ((b.ny + ty - 1) / ty);
    }
    if (take_alloc_failure()) return fail(LOPE_ERR_ALLOC, "allocation refused (fail_alloc option)");
    cudaError_t e = cudaMallocHost(&plan->pinned, sizeof(BatchGrid) * n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    std::memcpy(plan->pinned, plan->host.data(), sizeof(BatchGrid) * n);
    char* ws = static_cast<char*>(workspace);
    plan->dev.grids = reinterpret_cast<const BatchGrid*>(ws + 256);
    plan->dev.items = reinterpret_cast<BatchItem*>(ws + 256 + round256(sizeof(BatchGrid) * n));
    if (mode == 1 && items != batch_tb2_items(n, grids))
      return fail(LOPE_ERR_INVALID, "batch tile count mismatch");
    plan->dev.ngrids = n;
    plan->dev.nitems = items;
    plan->dev.tile_x = tx;
    plan->dev.tile_y = ty;
    plan->dev.ksteps = k;
    plan->dev.nsteps = nsteps;
    plan->dev.barrier = reinterpret_cast<unsigned int*>(ws);
    plan->dev.claim = reinterpret_cast<unsigned long long*>(ws + 128);
    plan->dev.err = d->err;
    plan->dev.wait_ns = (unsigned long long)wait_ms * 1000000ull;
    plan->dev.skip_block = int(skip);
    plan->dev.mode = mode;
    plan->blocks = std::min(items, maxb);
    // Capture: descriptor upload, barrier reset, persistent kernel.
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(d->capture, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    g_capturing = true;
    g_captured = 0;
    cudaError_t e1 = cudaMemcpyAsync(ws + 256, plan->pinned, sizeof(BatchGrid) * n,
                                     cudaMemcpyHostToDevice, d->capture);
    cudaError_t e2 = cudaMemsetAsync(ws, 0, 256, d->capture);
    cudaError_t e3 = launch_batch(plan->dev, s, dtype, plan->blocks, d->capture);
    g_capturing = false;
    e = cudaStreamEndCapture(d->capture, &graph);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(e3 != cudaSuccess ? e3 : e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e,
                       "capturing the batched launch");
    }
    e = cudaGraphInstantiate(&plan->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(batch)");
    plan->kernels = g_captured;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (g_batch.size() > 64) g_batch.clear();
    g_batch[key] = plan;
  }
  cudaError_t e = cudaGraphLaunch(plan->exec, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch(batch)");
  count_launches(plan->kernels);
  return LOPE_OK;
}

lope_status lope_autotune_batch(int n, const lope_grid* const* grids, const lope_stencil* stencil,
                                const void* const* in, void* const* out, void* const* work,
                                int64_t nsteps, void* workspace, size_t workspace_bytes,
                                lope_launch* best, double* best_ms, void* cuda_stream) {
  if (n < 1 || !grids || !stencil) return fail(LOPE_ERR_INVALID, "NULL argument");
  if (nsteps < 1) return fail(LOPE_ERR_INVALID, "autotune needs nsteps >= 1");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int tiles[][2] = {{128, 32}, {64, 32}, {128, 16}, {64, 16}};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double bms = 1e300;
  lope_launch bl = {0, 0, 0, 0, 0};
  lope_status last = LOPE_OK;
  std::vector<lope_launch> cands = {{kPathTma, kBatchTb2X, kBatchTb2Y, 2, -1}};
  for (const auto& t : tiles)
    for (int k : {1, 2, 4, 5}) cands.push_back({kPathTrap, t[0], t[1], k, -1});
  for (const auto& c : cands) {
    // first call builds and caches the plan's graph; the second is timed
    if ((last = lope_apply_batch(n, grids, stencil, in, out, work, nsteps, &c, workspace,
                                 workspace_bytes, cuda_stream)) != LOPE_OK)
      continue;
    cudaEventRecord(e0, st);
    last = lope_apply_batch(n, grids, stencil, in, out, work, nsteps, &c, workspace,
                            workspace_bytes, cuda_stream);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || last != LOPE_OK) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < bms) {
      bms = ms;
      bl = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (bl.path == 0) return last != LOPE_OK ? last : fail(LOPE_ERR_UNSUPPORTED, "no batched plan ran");
  g_last_error = "no error";
  {
    std::lock_guard<std::mutex> lk(g_btune_mu);
    g_btune[batch_sig(n, grids, stencil->s)] = {bl.path, bl.tile_x, bl.tile_y, bl.tsteps};
  }
  if (best) *best = bl;
  if (best_ms) *best_ms = bms;
  return LOPE_OK;
}

lope_status lope_workspace_size(const lope_grid* grid, const lope_stencil* stencil, int64_t nsteps,
                                int64_t checkpoint_every, size_t* bytes) {
  lope_status rs = check_linear_for_adjoint(grid, stencil);
  if (rs != LOPE_OK) return rs;
  if (nsteps < 1 || checkpoint_every < 1 || !bytes) return fail(LOPE_ERR_INVALID, "bad argument");
  *bytes = adj_layout(grid->g, nsteps, checkpoint_every).total;
  return LOPE_OK;
}

lope_status lope_forward_ckpt(const lope_grid* grid, const lope_stencil* stencil, const void* u0,
                              void* uT, int64_t nsteps, int64_t checkpoint_every, void* workspace,
                              size_t workspace_bytes, void* cuda_stream) {
  lope_status rs = check_linear_for_adjoint(grid, stencil);
  if (rs != LOPE_OK) return rs;
  if (nsteps < 1 || checkpoint_every < 1) return fail(LOPE_ERR_INVALID, "bad step counts");
  if (!u0 || !uT || !workspace || !aligned16(workspace)) return fail(LOPE_ERR_INVALID, "bad pointer");
  const AdjLayout L = adj_layout(grid->g, nsteps, checkpoint_every);
  if (workspace_bytes < L.total) return fail(LOPE_ERR_ALLOC, "workspace too small");
  char* ws = static_cast<char*>(workspace);
  return run_graph(adjoint_key(0, grid, stencil, {u0, uT, workspace}, nsteps, checkpoint_every),
                   static_cast<cudaStream_t>(cuda_stream), [&](cudaStream_t cs) {
                     return forward_ckpt_impl(grid, stencil, u0, uT, nsteps, checkpoint_every, ws,
                                              L, cs);
                   });
}

lope_status lope_vjp(const lope_grid* grid, const lope_stencil* stencil, const void* u0,
                     const void* grad_uT, int64_t nsteps, int64_t checkpoint_every,
                     int reuse_checkpoints, void* grad_u0, double* grad_coeff_dev, void* workspace,
                     size_t workspace_bytes, void* cuda_stream) {
  lope_status rs = check_linear_for_adjoint(grid, stencil);
  if (rs != LOPE_OK) return rs;
  if (nsteps < 1 || checkpoint_every < 1) return fail(LOPE_ERR_INVALID, "bad step counts");
  if (!u0 || !grad_uT || !grad_u0 || !workspace || !aligned16(workspace) || !aligned16(grad_u0) ||
      !aligned16(grad_uT))
    return fail(LOPE_ERR_INVALID, "bad pointer");
  const AdjLayout L = adj_layout(grid->g, nsteps, checkpoint_every);
  if (workspace_bytes < L.total) return fail(LOPE_ERR_ALLOC, "workspace too small");
  DevState* d = nullptr;
  if ((rs = dev_state(&d)) != LOPE_OK) return rs;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  char* ws = static_cast<char*>(workspace);
  const GraphKey key = adjoint_key(reuse_checkpoints ? 1 : 2, grid, stencil,
                                   {u0, grad_uT, grad_u0, grad_coeff_dev, workspace}, nsteps,
                                   checkpoint_every);
  return run_graph(key, st, [&](cudaStream_t cs) {
    if (!reuse_checkpoints) {
      // u_T itself is not needed; it lands in the last checkpoint slot.
      void* uT = ws + L.off_ckpt + size_t(L.nseg - 1) * L.field;
      lope_status r = forward_ckpt_impl(grid, stencil, u0, uT, nsteps, checkpoint_every, ws, L, cs);
      if (r != LOPE_OK) return r;
    }
    return reverse_impl(grid, stencil, u0, grad_uT, nsteps, checkpoint_every, grad_u0,
                        grad_coeff_dev, ws, L, d->err, cs);
  });
}

lope_status lope_adjoint(const lope_grid* grid, const lope_stencil* stencil, const void* u0,
                         const void* target, int64_t nsteps, int64_t checkpoint_every,
                         void* grad_u0, double* grad_coeff, double* loss, void* workspace,
                         size_t workspace_bytes, void* cuda_stream) {
  lope_status rs = check_linear_for_adjoint(grid, stencil);
  if (rs != LOPE_OK) return rs;
  if (nsteps < 1 || checkpoint_every < 1) return fail(LOPE_ERR_INVALID, "bad step counts");
  if (!u0 || !target || !grad_u0 || !workspace || !aligned16(workspace) || !aligned16(grad_u0))
    return fail(LOPE_ERR_INVALID, "bad pointer");
  const AdjLayout L = adj_layout(grid->g, nsteps, checkpoint_every);
  if (workspace_bytes < L.total) return fail(LOPE_ERR_ALLOC, "workspace too small");
  DevState* d = nullptr;
  if ((rs = dev_state(&d)) != LOPE_OK) return rs;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  char* ws = static_cast<char*>(workspace);
  double* scal = reinterpret_cast<double*>(ws + L.off_scal);
  rs = run_graph(adjoint_key(3, grid, stencil, {u0, target, grad_u0, workspace}, nsteps,
                             checkpoint_every),
                 st, [&](cudaStream_t cs) {
                   void* uT = ws + L.off_ckpt + size_t(L.nseg - 1) * L.field;
                   lope_status r = forward_ckpt_impl(grid, stencil, u0, uT, nsteps,
                                                     checkpoint_every, ws, L, cs);
                   if (r != LOPE_OK) return r;
                   double* partials = reinterpret_cast<double*>(ws + L.off_part);
                   void* lamT = ws + L.off_tmp;  // the forward work buffer is free now
                   cudaError_t e = launch_loss_seed(grid->g.dtype, uT, target, lamT,
                                                    npts(grid->g), partials, &scal[0], cs);
                   if (e != cudaSuccess) return cuda_fail(e, "loss kernel");
                   return reverse_impl(grid, stencil, u0, lamT, nsteps, checkpoint_every, grad_u0,
                                       &scal[1], ws, L, d->err, cs);
                 });
  if (rs != LOPE_OK) return rs;
  double host[2] = {0.0, 0.0};
  cudaError_t e = cudaMemcpyAsync(host, scal, sizeof(host), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "reading loss and dL/dc");
  if (loss) *loss = host[0];
  if (grad_coeff) *grad_coeff = host[1];
  if (!std::isfinite(host[0]) || !std::isfinite(host[1]))
    return fail(LOPE_ERR_NUMERIC, "non-finite loss or dL/dc");
  return LOPE_OK;
}

size_t lope_reduce_scratch_bytes(void) { return size_t(kReduceBlocks) * sizeof(double); }

lope_status lope_reduce(int op, lope_dtype dtype, const void* x, const void* y, int64_t n,
                        double* result_dev, void* scratch, void* cuda_stream) {
  if ((op != 0 && op != 1) || !x || (op == 1 && !y) || !result_dev || !scratch || n < 0)
    return fail(LOPE_ERR_INVALID, "bad reduction argument");
  if (dtype != LOPE_F64 && dtype != LOPE_F32 && dtype != LOPE_BF16)
    return fail(LOPE_ERR_INVALID, "unknown dtype");
  cudaError_t e = launch_reduce(op, dtype, x, y, n, static_cast<double*>(scratch), result_dev,
                                static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(e, "reduction kernel");
  return LOPE_OK;
}

lope_status lope_set_option(const char* name, int64_t value) {
  if (!name) return fail(LOPE_ERR_INVALID, "NULL option name");
  const std::string n(name);
  if (n == "wait_limit_ms") {
    if (value < 1 || value > 600000) return fail(LOPE_ERR_INVALID, "wait_limit_ms out of range");
    g_wait_limit_ms = value;
    return LOPE_OK;
  }
  if (n == "fail_alloc") {
    if (value < 0 || value > 1000000) return fail(LOPE_ERR_INVALID, "fail_alloc out of range");
    g_fail_alloc = value;
    return LOPE_OK;
  }
  if (n == "log") {
    if (value < 0 || value > 1) return fail(LOPE_ERR_INVALID, "log must be 0 or 1");
    g_log = int(value);
    return LOPE_OK;
  }
  if (n == "batch_skip_arrive") {
    if (value < -1 || value > (int64_t(1) << 30)) return fail(LOPE_ERR_INVALID, "bad block index");
    g_skip_arrive = value;
    return LOPE_OK;
  }
  return fail(LOPE_ERR_INVALID, "unknown option");
}

lope_status lope_sync_status(void* cuda_stream) {
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  DevState* d = nullptr;
  lope_status rs = dev_state(&d);
  if (rs != LOPE_OK) return rs;
  int flag = 0;
  e = cudaMemcpy(&flag, d->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device error flag");
  if (flag) {
    cudaMemset(d->err, 0, sizeof(int));
    if (flag == kErrHalo)
      return fail(LOPE_ERR_INVALID,
                  "a run-time compiled local function read outside its declared halo (the read "
                  "was clamped; Sec. 3.5 allows no out-of-bounds indexing)");
    return fail(LOPE_ERR_TIMEOUT, "a bounded in-kernel wait gave up");
  }
  return LOPE_OK;
}


lope_status lope_tune_cache_save(const char* path, const char* gpu_name) {
  if (!path) return fail(LOPE_ERR_INVALID, "NULL cache file path");
  std::string gpu;
  lope_status rs = gpu_tag_of(gpu_name, &gpu);
  if (rs != LOPE_OK) return rs;
  std::ostringstream os;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& kv : g_tune) {
      const TuneKey& k = kv.first;
      const Choice& c = kv.second;
      if (std::get<11>(k) != 0) continue;
      os << "lope-tune 1 " << gpu << " grid " << std::get<0>(k) << ' ' << std::get<1>(k) << ' '
         << std::get<2>(k) << ' ' << std::get<3>(k) << ' ' << std::get<4>(k) << ' ' << std::get<5>(k)
         << ' ' << std::get<6>(k) << ' ' << std::get<7>(k) << ' ' << std::get<8>(k) << ' '
         << std::get<9>(k) << ' ' << std::get<10>(k) << " : " << c.path << ' ' << c.tile_x << ' '
         << c.tile_y << ' ' << c.k << '\n';
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_btune_mu);
    for (const auto& kv : g_btune) {
      if (kv.first[5] != 0) continue;
      os << "lope-tune 1 " << gpu << " batch " << kv.first.size();
      for (int64_t v : kv.first) os << ' ' << v;
      const Choice& c = kv.second;
      os << " : " << c.path << ' ' << c.tile_x << ' ' << c.tile_y << ' ' << c.k << '\n';
    }
  }
  FILE* fp = std::fopen(path, "w");
  if (!fp) return fail(LOPE_ERR_INVALID, "cannot open the tune cache file for writing");
  const std::string text = os.str();
  const bool ok = std::fwrite(text.data(), 1, text.size(), fp) == text.size();
  if (std::fclose(fp) != 0 || !ok) return fail(LOPE_ERR_INVALID, "error writing the tune cache file");
  return LOPE_OK;
}

lope_status lope_tune_cache_load(const char* path, const char* gpu_name, int* loaded) {
  if (loaded) *loaded = 0;
  if (!path) return fail(LOPE_ERR_INVALID, "NULL cache file path");
  std::string gpu;
  lope_status rs = gpu_tag_of(gpu_name, &gpu);
  if (rs != LOPE_OK) return rs;
  std::ifstream in(path);
  if (!in) return fail(LOPE_ERR_INVALID, "cannot open the tune cache file");
  std::string line;
  int count = 0;
  while (std::getline(in, line)) {
    bool batch = false;
    TuneKey gk;
    BatchSig bk;
    Choice c;
    if (!parse_tune_line(line, gpu, &batch, &gk, &bk, &c)) continue;
    if (batch) {
      std::lock_guard<std::mutex> lk(g_btune_mu);
      g_btune[bk] = c;
    } else {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[gk] = c;
    }
    ++count;
  }
  if (loaded) *loaded = count;
  return LOPE_OK;
}

}  // extern "C"
