// Kernels for any grid shape, alignment and stencil shape (templates shared by
// k_generic.cu, plain sweeps, and k_generic_rk.cu, multi-stage forms):
//  * trap2d_kernel — shared-memory trapezoid tiles with temporal blocking
//    (2D; box stencils with corners allowed; see trap.cuh);
//  * trap2d_rk_kernel — the same tiles running fused Runge-Kutta steps;
//  * direct_kernel — one thread per output point reading its halo straight
//    from global memory through the boundary rule (2D and 3D).  This is the
//    plainest GPU form of "call the local function for each interior index"
//    (Sec. 2.2, Sec. 3.2) and serves shapes the TMA path cannot take.
#pragma once

#include <algorithm>

#include "trap.cuh"

namespace lope {

namespace {

// ------------------------------------------------------------------ trapezoid
template <class Op, class T>
__global__ void __launch_bounds__(256) trap2d_kernel(Op op, TrapGrid g, const T* __restrict__ in0,
                                                     const T* __restrict__ in1,
                                                     const T* __restrict__ in2, T* out0, T* out1,
                                                     T* out2, int TX, int TY, int k) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const T* src[3] = {in0, in1, in2};
  T* dst[3] = {out0, out1, out2};
  const int tiles_x = (g.nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
  trap_tile<Op, T>(op, src, dst, g, x0, y0, TX, TY, k, reinterpret_cast<C_t<T>*>(smem_raw));
}

// Multi-stage steps fused per tile (see trap_tile_rk).
template <class Op, class T>
__global__ void __launch_bounds__(256) trap2d_rk_kernel(Op op, TrapGrid g, const T* __restrict__ in0,
                                                        const T* __restrict__ in1,
                                                        const T* __restrict__ in2, T* out0, T* out1,
                                                        T* out2, int TX, int TY, int k, int stages) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const T* src[3] = {in0, in1, in2};
  T* dst[3] = {out0, out1, out2};
  const int tiles_x = (g.nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
  trap_tile_rk<Op, T>(op, src, dst, g, x0, y0, TX, TY, k, stages,
                      reinterpret_cast<C_t<T>*>(smem_raw));
}

TrapGrid trap_grid(const Geom& g) {
  TrapGrid t;
  t.nx = int(g.n[2]);
  t.ny = int(g.n[1]);
  for (int sd = 0; sd < 2; ++sd) {
    t.bc[0][sd] = g.bc[1][sd];
    t.bval[0][sd] = g.bval[1][sd];
    t.bc[1][sd] = g.bc[2][sd];
    t.bval[1][sd] = g.bval[2][sd];
  }
  return t;
}

// Multi-stage steps fused per tile (k_generic_rk.cu instantiates these).
template <class Op, class T>
cudaError_t run_trap_rk(const StepArgs& a, const Op& op) {
  const int TX = a.tile_x > 0 ? a.tile_x : 64, TY = a.tile_y > 0 ? a.tile_y : 32;
  const int k = std::max(1, a.ksteps);
  const int stages = a.s.stages;
  const TrapGrid g = trap_grid(a.g);
  const size_t smem = trap_smem_bytes(a.g.dtype, Op::NF, TX, TY, Op::R * k * stages, stages);
  {
    auto kern = &trap2d_rk_kernel<Op, T>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    const int blocks = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    const T* in[3] = {nullptr, nullptr, nullptr};
    T* out[3] = {nullptr, nullptr, nullptr};
    for (int f = 0; f < Op::NF; ++f) {
      in[f] = static_cast<const T*>(a.in[f]);
      out[f] = static_cast<T*>(a.out[f]);
    }
    kern<<<blocks, 256, smem, a.stream>>>(op, g, in[0], in[1], in[2], out[0], out[1], out[2], TX,
                                          TY, k, stages);
    count_launches(1);
    return cudaGetLastError();
  }
}

template <class Op, class T>
cudaError_t run_trap(const StepArgs& a, const Op& op) {
  const int TX = a.tile_x > 0 ? a.tile_x : 64, TY = a.tile_y > 0 ? a.tile_y : 32;
  const int k = std::max(1, a.ksteps);
  const TrapGrid g = trap_grid(a.g);
  const size_t smem = trap_smem_bytes(a.g.dtype, Op::NF, TX, TY, Op::R * k);
  auto kern = &trap2d_kernel<Op, T>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  const int blocks = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
  const T* in[3] = {nullptr, nullptr, nullptr};
  T* out[3] = {nullptr, nullptr, nullptr};
  for (int f = 0; f < Op::NF; ++f) {
    in[f] = static_cast<const T*>(a.in[f]);
    out[f] = static_cast<T*>(a.out[f]);
  }
  kern<<<blocks, 256, smem, a.stream>>>(op, g, in[0], in[1], in[2], out[0], out[1], out[2], TX, TY, k);
  count_launches(1);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ direct
template <class T, int NF>
struct GlobalAcc {
  using C = C_t<T>;
  const T* const* f;
  Geom g;
  int64_t z, y, x;
  __device__ __forceinline__ C operator()(int fi, int dx, int dy, int dz) const {
    int64_t q[3] = {z + dz, y + dy, x + dx};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if (q[ax] < 0 && g.bc[ax][0] == kDirichlet) return C(g.bval[ax][0]);
      if (q[ax] >= g.n[ax] && g.bc[ax][1] == kDirichlet) return C(g.bval[ax][1]);
    }
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int64_t m = g.n[ax];
      q[ax] = q[ax] < 0 ? q[ax] + m * ((-q[ax] + m - 1) / m) : q[ax] % m;
    }
    return to_c(__ldg(f[fi] + (q[0] * g.n[1] + q[1]) * g.n[2] + q[2]));
  }
  __device__ __forceinline__ int64_t gidx() const { return (z * g.n[1] + y) * g.n[2] + x; }
};

template <class Op, class T>
__global__ void __launch_bounds__(256) direct_kernel(Op op, Geom g, const T* in0, const T* in1,
                                                     const T* in2, T* out0, T* out1, T* out2,
                                                     double* partials) {
  using C = C_t<T>;
  const T* src[3] = {in0, in1, in2};
  T* dst[3] = {out0, out1, out2};
  const int64_t n = g.n[0] * g.n[1] * g.n[2];
  double red = 0.0;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < n;
       p += int64_t(gridDim.x) * blockDim.x) {
    GlobalAcc<T, Op::NF> acc{src, g, p / (g.n[1] * g.n[2]), (p / g.n[2]) % g.n[1], p % g.n[2]};
    C o[Op::NF];
    C r1 = C(0);
    op(acc, o, r1);
    red += double(r1);
#pragma unroll
    for (int f = 0; f < Op::NF; ++f) dst[f][p] = from_c<T>(o[f]);
  }
  if (Op::REDUCES) {
    __shared__ double ws[8];
    for (int o = 16; o > 0; o >>= 1) red += __shfl_down_sync(0xffffffffu, red, o);
    if (threadIdx.x % 32 == 0) ws[threadIdx.x / 32] = red;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < int(blockDim.x / 32); ++w) s += ws[w];
      partials[blockIdx.x] += s;
    }
  }
}

int direct_grid(const Geom& g) {
  const int64_t n = g.n[0] * g.n[1] * g.n[2];
  return int(std::min<int64_t>((n + 255) / 256, 152 * 8));
}

template <class Op, class T>
cudaError_t run_direct(const StepArgs& a, const Op& op, int* blocks_out) {
  const int blocks = direct_grid(a.g);
  if (blocks_out) *blocks_out = blocks;
  if (Op::REDUCES && (!a.partials || blocks > a.partial_count)) return cudaErrorInvalidValue;
  const T* in[3] = {nullptr, nullptr, nullptr};
  T* out[3] = {nullptr, nullptr, nullptr};
  for (int f = 0; f < Op::NF; ++f) {
    in[f] = static_cast<const T*>(a.in[f]);
    out[f] = static_cast<T*>(a.out[f]);
  }
  direct_kernel<Op, T><<<blocks, 256, 0, a.stream>>>(op, a.g, in[0], in[1], in[2], out[0], out[1],
                                                      out[2], a.partials);
  count_launches(1);
  return cudaGetLastError();
}

// RK = false: plain sweeps (trapezoid with temporal blocking, direct).  RK =
// true: the multi-stage forms (fused trapezoid steps; a combining stage on the
// direct kernel, out = a * base + b * E(in)).
template <bool RK, class Op, class T>
cudaError_t run_any(const StepArgs& a, const Op& op, bool trap, int* blocks) {
  if (trap) {
    if constexpr (Op::NDIM == 2 && !Op::REDUCES) {
      if constexpr (RK) return run_trap_rk<Op, T>(a, op);
      else return run_trap<Op, T>(a, op);
    }
    return cudaErrorNotSupported;
  }
  if constexpr (RK) {
    if constexpr (!Op::REDUCES) {
      OpStage<Op, T> st;
      st.op = op;
      st.a = a.rk_a;
      st.b = a.rk_b;
      for (int f = 0; f < kMaxFields; ++f) st.base[f] = static_cast<const T*>(a.base[f]);
      return run_direct<OpStage<Op, T>, T>(a, st, blocks);
    }
    return cudaErrorNotSupported;
  } else {
    return run_direct<Op, T>(a, op, blocks);
  }
}

template <int ND, int RR> OpStarLinear<ND, RR> star_op(const StencilDesc& s) {
  OpStarLinear<ND, RR> op;
  for (int ax = 0; ax < 3; ++ax)
    for (int d = 0; d < 2 * RR + 1; ++d) op.w[ax][d] = s.star_w[ax][d];
  return op;
}
template <int ND, int RR> OpBoxLinear<ND, RR> box_op(const StencilDesc& s) {
  OpBoxLinear<ND, RR> op;
  for (int i = 0; i < OpBoxLinear<ND, RR>::ZS * (2 * RR + 1) * (2 * RR + 1); ++i) op.w[i] = s.box[i];
  return op;
}

template <bool RK, class T> cudaError_t dispatch_t(const StepArgs& a, bool trap, int* blocks) {
  const StencilDesc& s = a.s;
  if (!RK && a.adjoint) {
    switch (s.kind) {
      case kJacobi5: return run_any<RK, OpAdjDiffusion<kJacobi5, T>, T>(a, {s.prm[0], (const T*)a.ut}, trap, blocks);
      case kStar9r2: return run_any<RK, OpAdjDiffusion<kStar9r2, T>, T>(a, {s.prm[0], (const T*)a.ut}, trap, blocks);
      case kDiff7: return run_any<RK, OpAdjDiffusion<kDiff7, T>, T>(a, {s.prm[0], (const T*)a.ut}, trap, blocks);
      default: break;
    }
  }
  switch (s.kind) {
    case kJacobi5: return run_any<RK, OpJacobi5, T>(a, {s.prm[0]}, trap, blocks);
    case kStar9r2: return run_any<RK, OpStar9r2, T>(a, {s.prm[0]}, trap, blocks);
    case kDiff7: return run_any<RK, OpDiff7, T>(a, {s.prm[0]}, trap, blocks);
    case kSwe: return run_any<RK, OpSwe, T>(a, {-s.prm[0] * s.prm[2], -s.prm[0] * s.prm[1]}, trap, blocks);
    case kSweFlux: return run_any<RK, OpSweFlux, T>(a, OpSweFlux::make(s.prm), trap, blocks);
    case kLinear:
      if (s.star) {
        if (s.ndim == 2 && s.radius == 1) return run_any<RK, OpStarLinear<2, 1>, T>(a, star_op<2, 1>(s), trap, blocks);
        if (s.ndim == 2 && s.radius == 2) return run_any<RK, OpStarLinear<2, 2>, T>(a, star_op<2, 2>(s), trap, blocks);
        if (s.ndim == 3 && s.radius == 1) return run_any<RK, OpStarLinear<3, 1>, T>(a, star_op<3, 1>(s), trap, blocks);
        if (s.ndim == 3 && s.radius == 2) return run_any<RK, OpStarLinear<3, 2>, T>(a, star_op<3, 2>(s), trap, blocks);
      } else {
        if (s.ndim == 2 && s.radius == 1) return run_any<RK, OpBoxLinear<2, 1>, T>(a, box_op<2, 1>(s), trap, blocks);
        if (s.ndim == 2 && s.radius == 2) return run_any<RK, OpBoxLinear<2, 2>, T>(a, box_op<2, 2>(s), trap, blocks);
        if (s.ndim == 3 && s.radius == 1) return run_any<RK, OpBoxLinear<3, 1>, T>(a, box_op<3, 1>(s), trap, blocks);
        if (s.ndim == 3 && s.radius == 2) return run_any<RK, OpBoxLinear<3, 2>, T>(a, box_op<3, 2>(s), trap, blocks);
      }
      return cudaErrorNotSupported;
    default: return cudaErrorNotSupported;
  }
}

template <bool RK> cudaError_t dispatch_generic(const StepArgs& a, bool trap, int* blocks) {
  switch (a.g.dtype) {
    case kF32: return dispatch_t<RK, float>(a, trap, blocks);
    case kF64: return dispatch_t<RK, double>(a, trap, blocks);
    case kBF16: return dispatch_t<RK, __nv_bfloat16>(a, trap, blocks);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace
}  // namespace lope
