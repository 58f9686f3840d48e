// TMA kernel dispatch for the combining stages of the multi-stage (Runge-Kutta)
// schemes: the same TMA tiles / z-march as a plain sweep, with the local
// function wrapped in OpStage (out = a * base + b * E(in), base read at the
// local element only).  Compiled as its own translation unit so that these
// instances build in parallel with the plain ones.
#include "tma_kernels.cuh"

namespace lope {

namespace {

template <class Op, class T, int RANK>
cudaError_t run_stage(const StepArgs& a, const Op& op) {
  OpStage<Op, T> st;
  st.op = op;
  st.a = a.rk_a;
  st.b = a.rk_b;
  for (int f = 0; f < kMaxFields; ++f) st.base[f] = static_cast<const T*>(a.base[f]);
  return TmaRunner<OpStage<Op, T>, T, RANK>::run(a, st, nullptr);
}

template <int ND, int RR> OpStarLinear<ND, RR> star_op(const StencilDesc& s) {
  OpStarLinear<ND, RR> op;
  for (int ax = 0; ax < 3; ++ax)
    for (int d = 0; d < 2 * RR + 1; ++d) op.w[ax][d] = s.star_w[ax][d];
  return op;
}

template <int RR> OpBoxLinear<2, RR> box_op(const StencilDesc& s) {
  OpBoxLinear<2, RR> op;
  for (int i = 0; i < (2 * RR + 1) * (2 * RR + 1); ++i) op.w[i] = s.box[i];
  return op;
}

template <class T> cudaError_t dispatch_t(const StepArgs& a) {
  const StencilDesc& s = a.s;
  switch (s.kind) {
    case kJacobi5: return run_stage<OpJacobi5, T, 2>(a, {s.prm[0]});
    case kStar9r2: return run_stage<OpStar9r2, T, 2>(a, {s.prm[0]});
    case kDiff7: return run_stage<OpDiff7, T, 3>(a, {s.prm[0]});
    case kSwe: return run_stage<OpSwe, T, 2>(a, {-s.prm[0] * s.prm[2], -s.prm[0] * s.prm[1]});
    case kSweFlux: return run_stage<OpSweFlux, T, 2>(a, OpSweFlux::make(s.prm));
    case kLinear:
      if (!s.star) {
        if (s.ndim == 2 && s.radius == 1) return run_stage<OpBoxLinear<2, 1>, T, 2>(a, box_op<1>(s));
        if (s.ndim == 2 && s.radius == 2) return run_stage<OpBoxLinear<2, 2>, T, 2>(a, box_op<2>(s));
        return cudaErrorNotSupported;
      }
      if (s.ndim == 2 && s.radius == 1) return run_stage<OpStarLinear<2, 1>, T, 2>(a, star_op<2, 1>(s));
      if (s.ndim == 2 && s.radius == 2) return run_stage<OpStarLinear<2, 2>, T, 2>(a, star_op<2, 2>(s));
      if (s.ndim == 3 && s.radius == 1) return run_stage<OpStarLinear<3, 1>, T, 3>(a, star_op<3, 1>(s));
      if (s.ndim == 3 && s.radius == 2) return run_stage<OpStarLinear<3, 2>, T, 3>(a, star_op<3, 2>(s));
      return cudaErrorNotSupported;
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

cudaError_t launch_tma_stage(const StepArgs& a) {
  if (a.s.kind == kUser) return jit_launch(a, kPathTma);
  switch (a.g.dtype) {
    case kF32: return dispatch_t<float>(a);
    case kF64: return dispatch_t<double>(a);
    case kBF16: return dispatch_t<__nv_bfloat16>(a);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace lope
