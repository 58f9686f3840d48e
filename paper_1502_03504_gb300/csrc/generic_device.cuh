// Kernels for any grid shape, alignment and stencil shape (device templates;
// compiles under nvcc and NVRTC alike):
//  * trap2d_kernel — shared-memory trapezoid tiles with temporal blocking
//    (2D; box stencils with corners allowed; see trap.cuh);
//  * trap2d_rk_kernel — the same tiles running fused Runge-Kutta steps;
//  * direct_kernel — one thread per output point reading its halo straight
//    from global memory through the boundary rule (2D and 3D).  This is the
//    plainest GPU form of "call the local function for each interior index"
//    (Sec. 2.2, Sec. 3.2) and serves shapes the TMA path cannot take.
#pragma once

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

}  // namespace
}  // namespace lope
