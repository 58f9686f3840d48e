// Host-side runners of the kernels for any grid shape, alignment and stencil
// shape (the kernels are in generic_device.cuh), shared by k_generic.cu (plain
// sweeps) and k_generic_rk.cu (multi-stage forms):
//  * trap2d_kernel — shared-memory trapezoid tiles with temporal blocking
//    (2D; box stencils with corners allowed; see trap.cuh);
//  * trap2d_rk_kernel — the same tiles running fused Runge-Kutta steps;
//  * direct_kernel — one thread per output point reading its halo straight
//    from global memory through the boundary rule (2D and 3D).  This is the
//    plainest GPU form of "call the local function for each interior index"
//    (Sec. 2.2, Sec. 3.2) and serves shapes the TMA path cannot take.
#pragma once

#include <algorithm>
#include <type_traits>

#include "generic_device.cuh"
#include "tma_kernels.cuh"

namespace lope {

namespace {

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

// Blocks of the direct kernel: one per unit of 256 points of a row, at most
// eight per SM.
int direct_grid(const Geom& g) {
  const int64_t units = g.n[0] * g.n[1] * ((g.n[2] + 255) / 256);
  return int(std::min<int64_t>(units, 152 * 8));
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

// Plane march geometry: tx x ty column tiles; z cut into chunks of at least
// 16 planes so that about two waves of 256-thread blocks (per_sm per SM) are
// in flight (each chunk stages 2R extra planes).
inline bool march_geometry_t(const Geom& g, int tx, int ty, int per_sm, int* blocks, int* zchunk) {
  const int64_t tiles = ((g.n[2] + tx - 1) / tx) * ((g.n[1] + ty - 1) / ty);
  const int64_t slots = 2 * int64_t(per_sm) * 152;
  int64_t nzc = std::max<int64_t>(1, std::min<int64_t>(g.n[0] / 16, (slots + tiles - 1) / tiles));
  const int64_t zc = (g.n[0] + nzc - 1) / nzc;
  nzc = (g.n[0] + zc - 1) / zc;
  if (tiles * nzc > int64_t(0x7fffffff)) return false;
  *blocks = int(tiles * nzc);
  *zchunk = int(zc);
  return true;
}
// The same cut for the asynchronous march, counted in whole waves: among the
// chunk counts that keep 16 planes or more per chunk, the one that maximises
// the busy fraction of the last wave times the share of planes that are not
// halo (each chunk stages 2R planes twice).
inline bool march_chunks(const Geom& g, int tx, int ty, int R, int per_sm, int* blocks,
                         int* zchunk) {
  const int64_t tiles = ((g.n[2] + tx - 1) / tx) * ((g.n[1] + ty - 1) / ty);
  const int64_t conc = int64_t(per_sm) * 152;
  const int64_t most = std::max<int64_t>(1, std::min<int64_t>(g.n[0] / 16, 4 * conc / tiles + 1));
  double best = -1.0;
  int64_t bzc = g.n[0], bn = 1;
  for (int64_t n = 1; n <= most; ++n) {
    const int64_t zc = (g.n[0] + n - 1) / n, nzc = (g.n[0] + zc - 1) / zc;
    const int64_t b = tiles * nzc, waves = (b + conc - 1) / conc;
    const double score = double(b) / double(waves * conc) * double(zc) / double(zc + 2 * R);
    if (score > best + 1e-9) {
      best = score;
      bzc = zc;
      bn = nzc;
    }
  }
  if (tiles * bn > int64_t(0x7fffffff)) return false;
  *blocks = int(tiles * bn);
  *zchunk = int(bzc);
  return true;
}
inline bool march_geometry(const Geom& g, int* blocks, int* zchunk) {
  return march_geometry_t(g, kMarchX, kMarchY, 8, blocks, zchunk);
}

// Whether Op is a combining stage of a multi-stage step (it reads its base
// state at the output element, which the copied-plane march's pairs would
// read unaligned).
template <class Op> struct IsStage : std::false_type {};
template <class Op, class T> struct IsStage<OpStage<Op, T>> : std::true_type {};

// FP32 / FP64 grids: plain sweeps of star functions take the z-march with
// copied planes (ca3d_kernel: paired consumers, z register queues); box
// functions and combining stages the asynchronous-copy plane march (64 x 16
// tiles, four rows per thread).  BF16 grids take the register-staged plane
// march (widened on load).
template <class Op, class T>
cudaError_t run_march(const StepArgs& a, const Op& op) {
  const T* in[3] = {nullptr, nullptr, nullptr};
  T* out[3] = {nullptr, nullptr, nullptr};
  for (int f = 0; f < Op::NF; ++f) {
    in[f] = static_cast<const T*>(a.in[f]);
    out[f] = static_cast<T*>(a.out[f]);
  }
  int blocks = 0, zchunk = 0;
  if constexpr (sizeof(T) == sizeof(C_t<T>) && Op::STAR && !IsStage<Op>::value) {
    return CaRunner<Op, T>::run(a, op, [&](int tx, int ty, int per_sm, int* b, int* zc) {
      return march_chunks(a.g, tx, ty, Op::R, per_sm, b, zc);
    });
  } else if constexpr (sizeof(T) == sizeof(C_t<T>)) {
    constexpr int smem = march_async_smem<C_t<T>, Op::NF, Op::R>();
    auto kern = &march3d_async_kernel<Op, T>;
    static int per_sm = 0;  // resident blocks per SM, measured once per instance
    if (per_sm == 0) {
      if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
      }
      int n = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 256, smem);
      if (e != cudaSuccess) return e;
      per_sm = std::max(1, n);
    }
    if (!march_chunks(a.g, kAsyncX, kAsyncY, Op::R, per_sm, &blocks, &zchunk))
      return cudaErrorInvalidConfiguration;
    kern<<<blocks, 256, smem, a.stream>>>(op, a.g, in[0], in[1], in[2], out[0], out[1], out[2],
                                          zchunk);
  } else {
    if (!march_geometry(a.g, &blocks, &zchunk)) return cudaErrorInvalidConfiguration;
    march3d_plain_kernel<Op, T><<<blocks, 256, 0, a.stream>>>(op, a.g, in[0], in[1], in[2],
                                                               out[0], out[1], out[2], zchunk);
  }
  count_launches(1);
  return cudaGetLastError();
}

// RK = false: plain sweeps (trapezoid with temporal blocking, direct, column
// march).  RK = true: the multi-stage forms (fused trapezoid steps; a
// combining stage, out = a * base + b * E(in), on the direct kernel or the
// plane march).
template <bool RK, class Op, class T>
cudaError_t run_any(const StepArgs& a, const Op& op, int kind, int* blocks) {
  if (kind == kGenTrap) {
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
      if (kind == kGenMarch) {
        if constexpr (Op::NDIM == 3) return run_march<OpStage<Op, T>, T>(a, st);
        return cudaErrorNotSupported;
      }
      return run_direct<OpStage<Op, T>, T>(a, st, blocks);
    }
    return cudaErrorNotSupported;
  } else {
    if (kind == kGenMarch) {
      if constexpr (Op::NDIM == 3 && !Op::REDUCES) return run_march<Op, T>(a, op);
      return cudaErrorNotSupported;
    }
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

template <bool RK, class T> cudaError_t dispatch_t(const StepArgs& a, int kind, int* blocks) {
  const StencilDesc& s = a.s;
  if (!RK && a.adjoint) {
    switch (s.kind) {
      case kJacobi5: return run_any<RK, OpAdjDiffusion<kJacobi5, T>, T>(a, {s.prm[0], (const T*)a.ut}, kind, blocks);
      case kStar9r2: return run_any<RK, OpAdjDiffusion<kStar9r2, T>, T>(a, {s.prm[0], (const T*)a.ut}, kind, blocks);
      case kDiff7: return run_any<RK, OpAdjDiffusion<kDiff7, T>, T>(a, {s.prm[0], (const T*)a.ut}, kind, blocks);
      default: break;
    }
  }
  switch (s.kind) {
    case kJacobi5: return run_any<RK, OpJacobi5, T>(a, {s.prm[0]}, kind, blocks);
    case kStar9r2: return run_any<RK, OpStar9r2, T>(a, {s.prm[0]}, kind, blocks);
    case kDiff7: return run_any<RK, OpDiff7, T>(a, {s.prm[0]}, kind, blocks);
    case kSwe: return run_any<RK, OpSwe, T>(a, {-s.prm[0] * s.prm[2], -s.prm[0] * s.prm[1]}, kind, blocks);
    case kSweFlux: return run_any<RK, OpSweFlux, T>(a, OpSweFlux::make(s.prm), kind, blocks);
    case kLinear:
      if (s.star) {
        if (s.ndim == 2 && s.radius == 1) return run_any<RK, OpStarLinear<2, 1>, T>(a, star_op<2, 1>(s), kind, blocks);
        if (s.ndim == 2 && s.radius == 2) return run_any<RK, OpStarLinear<2, 2>, T>(a, star_op<2, 2>(s), kind, blocks);
        if (s.ndim == 3 && s.radius == 1) return run_any<RK, OpStarLinear<3, 1>, T>(a, star_op<3, 1>(s), kind, blocks);
        if (s.ndim == 3 && s.radius == 2) return run_any<RK, OpStarLinear<3, 2>, T>(a, star_op<3, 2>(s), kind, blocks);
      } else {
        if (s.ndim == 2 && s.radius == 1) return run_any<RK, OpBoxLinear<2, 1>, T>(a, box_op<2, 1>(s), kind, blocks);
        if (s.ndim == 2 && s.radius == 2) return run_any<RK, OpBoxLinear<2, 2>, T>(a, box_op<2, 2>(s), kind, blocks);
        if (s.ndim == 3 && s.radius == 1) return run_any<RK, OpBoxLinear<3, 1>, T>(a, box_op<3, 1>(s), kind, blocks);
        if (s.ndim == 3 && s.radius == 2) return run_any<RK, OpBoxLinear<3, 2>, T>(a, box_op<3, 2>(s), kind, blocks);
      }
      return cudaErrorNotSupported;
    default: return cudaErrorNotSupported;
  }
}

template <bool RK> cudaError_t dispatch_generic(const StepArgs& a, int kind, int* blocks) {
  switch (a.g.dtype) {
    case kF32: return dispatch_t<RK, float>(a, kind, blocks);
    case kF64: return dispatch_t<RK, double>(a, kind, blocks);
    case kBF16: return dispatch_t<RK, __nv_bfloat16>(a, kind, blocks);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace
}  // namespace lope
