// TMA kernel dispatch for plain sweeps of the local functions: picks the
// TmaRunner instance for the stencil kind and storage type (the kernels and
// the runner live in tma_kernels.cuh).
#include "tma_kernels.cuh"

namespace lope {

namespace {

template <class T> cudaError_t dispatch_t(const StepArgs& a, int* blocks) {
  const StencilDesc& s = a.s;
  if (a.adjoint) {
    switch (s.kind) {
      case kJacobi5: return TmaRunner<OpAdjDiffusion<kJacobi5, T>, T, 2>::run(a, {s.prm[0], (const T*)a.ut}, blocks);
      case kStar9r2: return TmaRunner<OpAdjDiffusion<kStar9r2, T>, T, 2>::run(a, {s.prm[0], (const T*)a.ut}, blocks);
      case kDiff7: return TmaRunner<OpAdjDiffusion<kDiff7, T>, T, 3>::run(a, {s.prm[0], (const T*)a.ut}, blocks);
      default: break;  // linear stencils: the caller passes reflected weights, no reduction
    }
  }
  if (a.ksteps == 2) {  // two sweeps per launch (temporal blocking)
    if (!tb2_supported(a)) return cudaErrorNotSupported;
    if (s.kind == kDiff7) return TmaRunner<OpDiff7, T, 3>::run_tb2(a, {s.prm[0]}, blocks);
    if (s.kind == kJacobi5) return TmaRunner<OpJacobi5, T, 2>::run_tb2(a, {s.prm[0]}, blocks);
    if (s.kind == kStar9r2) return TmaRunner<OpStar9r2, T, 2>::run_tb2(a, {s.prm[0]}, blocks);
    if (s.kind == kSwe)
      return TmaRunner<OpSwe, T, 2>::run_tb2(a, {-s.prm[0] * s.prm[2], -s.prm[0] * s.prm[1]}, blocks);
    if (s.kind == kSweFlux) return TmaRunner<OpSweFlux, T, 2>::run_tb2(a, OpSweFlux::make(s.prm), blocks);
    if (!s.star) {  // box tables (2D)
      if (s.radius == 1) {
        OpBoxLinear<2, 1> op;
        for (int i = 0; i < 9; ++i) op.w[i] = s.box[i];
        return TmaRunner<OpBoxLinear<2, 1>, T, 2>::run_tb2(a, op, blocks);
      }
      OpBoxLinear<2, 2> op;
      for (int i = 0; i < 25; ++i) op.w[i] = s.box[i];
      return TmaRunner<OpBoxLinear<2, 2>, T, 2>::run_tb2(a, op, blocks);
    }
    if (s.ndim == 3) {
      OpStarLinear<3, 1> op;
      for (int ax = 0; ax < 3; ++ax) for (int d = 0; d < 3; ++d) op.w[ax][d] = s.star_w[ax][d];
      return TmaRunner<OpStarLinear<3, 1>, T, 3>::run_tb2(a, op, blocks);
    }
    if (s.radius == 1) {
      OpStarLinear<2, 1> op;
      for (int ax = 0; ax < 3; ++ax) for (int d = 0; d < 3; ++d) op.w[ax][d] = s.star_w[ax][d];
      return TmaRunner<OpStarLinear<2, 1>, T, 2>::run_tb2(a, op, blocks);
    }
    OpStarLinear<2, 2> op;
    for (int ax = 0; ax < 3; ++ax) for (int d = 0; d < 5; ++d) op.w[ax][d] = s.star_w[ax][d];
    return TmaRunner<OpStarLinear<2, 2>, T, 2>::run_tb2(a, op, blocks);
  }
  switch (s.kind) {
    case kJacobi5: return TmaRunner<OpJacobi5, T, 2>::run(a, {s.prm[0]}, blocks);
    case kStar9r2: return TmaRunner<OpStar9r2, T, 2>::run(a, {s.prm[0]}, blocks);
    case kDiff7: return TmaRunner<OpDiff7, T, 3>::run(a, {s.prm[0]}, blocks);
    case kSwe: return TmaRunner<OpSwe, T, 2>::run(a, {-s.prm[0] * s.prm[2], -s.prm[0] * s.prm[1]}, blocks);
    case kSweFlux: return TmaRunner<OpSweFlux, T, 2>::run(a, OpSweFlux::make(s.prm), blocks);
    case kLinear: {
      if (!s.star) {  // box tables (2D): corner taps read the wide box
        if (s.ndim == 2 && s.radius == 1) {
          OpBoxLinear<2, 1> op;
          for (int i = 0; i < 9; ++i) op.w[i] = s.box[i];
          return TmaRunner<OpBoxLinear<2, 1>, T, 2>::run(a, op, blocks);
        }
        if (s.ndim == 2 && s.radius == 2) {
          OpBoxLinear<2, 2> op;
          for (int i = 0; i < 25; ++i) op.w[i] = s.box[i];
          return TmaRunner<OpBoxLinear<2, 2>, T, 2>::run(a, op, blocks);
        }
        return cudaErrorNotSupported;
      }
      if (s.ndim == 2 && s.radius == 1) {
        OpStarLinear<2, 1> op;
        for (int ax = 0; ax < 3; ++ax) for (int d = 0; d < 3; ++d) op.w[ax][d] = s.star_w[ax][d];
        return TmaRunner<OpStarLinear<2, 1>, T, 2>::run(a, op, blocks);
      }
      if (s.ndim == 2 && s.radius == 2) {
        OpStarLinear<2, 2> op;
        for (int ax = 0; ax < 3; ++ax) for (int d = 0; d < 5; ++d) op.w[ax][d] = s.star_w[ax][d];
        return TmaRunner<OpStarLinear<2, 2>, T, 2>::run(a, op, blocks);
      }
      if (s.ndim == 3 && s.radius == 1) {
        OpStarLinear<3, 1> op;
        for (int ax = 0; ax < 3; ++ax) for (int d = 0; d < 3; ++d) op.w[ax][d] = s.star_w[ax][d];
        return TmaRunner<OpStarLinear<3, 1>, T, 3>::run(a, op, blocks);
      }
      if (s.ndim == 3 && s.radius == 2) {
        OpStarLinear<3, 2> op;
        for (int ax = 0; ax < 3; ++ax) for (int d = 0; d < 5; ++d) op.w[ax][d] = s.star_w[ax][d];
        return TmaRunner<OpStarLinear<3, 2>, T, 3>::run(a, op, blocks);
      }
      return cudaErrorNotSupported;
    }
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

bool tma_supported(const StepArgs& a) {
  const Geom& g = a.g;
  const StencilDesc& s = a.s;
  if (a.ksteps == 2 && !tb2_supported(a)) return false;
  if (a.ksteps < 1 || a.ksteps > 2 || s.radius < 1 || s.radius > 2) return false;
  if ((s.kind == kSwe || s.kind == kSweFlux) && g.ndim != 2) return false;
  if (s.kind == kUser && (a.adjoint || !jit_tma_ok(static_cast<const JitProgram*>(s.jit)))) return false;
  if (!s.star && (g.ndim != 2 || a.adjoint)) return false;  // box stencils: 2D tiles only
  const int esz = g.dtype == kF64 ? 8 : g.dtype == kF32 ? 4 : 2;
  const int cw = 16 / esz;
  if ((g.n[2] * esz) % 16 != 0) return false;
  for (int ax = 0; ax < 3; ++ax) {
    if (g.n[ax] > (int64_t(1) << 30)) return false;
    for (int sd = 0; sd < 2; ++sd) {
      if (g.bc[ax][sd] == kDirichlet && g.bval[ax][sd] != 0.0 && !a.adjoint) return false;
      // an external halo: slowest axis, one sweep per launch (the caller
      // refreshes it between sweeps)
      if (g.bc[ax][sd] == kExternal && (ax != 3 - g.ndim || a.ksteps != 1 || a.adjoint))
        return false;
    }
    if (g.bc[ax][0] == kPeriodic && ax >= 3 - g.ndim && g.n[ax] < s.radius) return false;
  }
  if (g.bc[2][0] == kPeriodic && g.n[2] < cw) return false;
  for (int f = 0; f < g.nf; ++f)
    if ((reinterpret_cast<uintptr_t>(a.in[f]) & 15) != 0) return false;
  if (a.adjoint && s.kind == kLinear) return true;
  if (a.adjoint && s.kind != kJacobi5 && s.kind != kStar9r2 && s.kind != kDiff7) return false;
  return true;
}

cudaError_t launch_tma(const StepArgs& a, int* blocks) {
  if (a.s.kind == kUser) return jit_launch(a, kPathTma);
  switch (a.g.dtype) {
    case kF32: return dispatch_t<float>(a, blocks);
    case kF64: return dispatch_t<double>(a, blocks);
    case kBF16: return dispatch_t<__nv_bfloat16>(a, blocks);
    default: return cudaErrorNotSupported;
  }
}

int tma_blocks(const StepArgs& a) {
  // Number of blocks the adjoint kernels use, for sizing partial sums.
  int b = 0;
  auto pick = [&](auto tag) {
    using T = decltype(tag);
    TmaParams<OpAdjDiffusion<kDiff7, T>, T> p3;
    TmaParams<OpAdjDiffusion<kJacobi5, T>, T> p2;
    TmaParams<OpAdjDiffusion<kStar9r2, T>, T> p2b;
    if (a.g.ndim == 3) TmaRunner<OpAdjDiffusion<kDiff7, T>, T, 3>::geometry(a, p3, &b);
    else if (a.s.kind == kStar9r2) TmaRunner<OpAdjDiffusion<kStar9r2, T>, T, 2>::geometry(a, p2b, &b);
    else TmaRunner<OpAdjDiffusion<kJacobi5, T>, T, 2>::geometry(a, p2, &b);
  };
  if (a.g.dtype == kF32) pick(float());
  else if (a.g.dtype == kF64) pick(double());
  else pick(__nv_bfloat16());
  return b;
}

}  // namespace lope
