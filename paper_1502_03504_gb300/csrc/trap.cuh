// Shared-memory trapezoid tile with temporal blocking, used by the per-grid
// trapezoid kernel (k_generic.cu) and by the persistent batched kernel
// (k_batch.cu), so both evaluate exactly the same arithmetic.
//
// A block stages a (TY + 2Rk) x (TX + 2Rk) window of the state, filling every
// cell from the boundary rule (periodic wrap or Dirichlet value; Sec. 2.2
// "Halo regions", Sec. 3.2 BC=CYCLIC), then runs k sweeps of the local
// function inside shared memory.  Sweep s updates the window shrunk by s*R on
// each side from the frozen result of sweep s-1 (the snapshot semantics of
// Sec. 2.2 / Sec. 3.5), so after k sweeps the central TX x TY tile holds the
// state k steps later.  Fusing k sweeps per pass is the "compiler fuses the
// small functions" latitude of Sec. 3.5.  Every sweep rounds to the storage
// precision, so the result is bitwise the same for any k and tile shape.
#pragma once

#include "device_common.cuh"

namespace lope {

struct TrapGrid {
  int nx, ny;
  int bc[2][2];        // [0 = y axis, 1 = x axis][side]
  double bval[2][2];
};

template <class C, int NF>
struct TrapAcc {
  const C* buf;  // NF planes of H x W
  int W, HW;
  int i, j;
  __device__ __forceinline__ C operator()(int f, int dx, int dy, int) const {
    return buf[f * HW + (j + dy) * W + (i + dx)];
  }
  __device__ __forceinline__ int64_t gidx() const { return 0; }
};

// Value of the state at global (gy, gx), which may lie outside the grid.
template <class T>
__device__ __forceinline__ C_t<T> halo_read(const T* src, const TrapGrid& g, int gy, int gx) {
  using C = C_t<T>;
  if (gy < 0 && g.bc[0][0] == kDirichlet) return C(g.bval[0][0]);
  if (gy >= g.ny && g.bc[0][1] == kDirichlet) return C(g.bval[0][1]);
  if (gx < 0 && g.bc[1][0] == kDirichlet) return C(g.bval[1][0]);
  if (gx >= g.nx && g.bc[1][1] == kDirichlet) return C(g.bval[1][1]);
  gy = wrap(gy, g.ny);
  gx = wrap(gx, g.nx);
  return to_c(__ldcg(src + int64_t(gy) * g.nx + gx));
}

// Dirichlet cells outside the grid keep their halo value in every sweep.
__device__ __forceinline__ bool outside_dirichlet(const TrapGrid& g, int gy, int gx, double* v) {
  if (gy < 0 && g.bc[0][0] == kDirichlet) { *v = g.bval[0][0]; return true; }
  if (gy >= g.ny && g.bc[0][1] == kDirichlet) { *v = g.bval[0][1]; return true; }
  if (gx < 0 && g.bc[1][0] == kDirichlet) { *v = g.bval[1][0]; return true; }
  if (gx >= g.nx && g.bc[1][1] == kDirichlet) { *v = g.bval[1][1]; return true; }
  return false;
}

// Stage the window cell at global (gy, gx) into `cell`: the Dirichlet value
// past a Dirichlet side (stored directly), else the element at the wrapped
// position.  Where the stored and computed types agree (FP32, FP64) the
// element moves by an asynchronous copy, so a thread keeps every copy of the
// window in flight at once; the caller ends the fill with cp_async_wait_all
// and a block barrier.  BF16 is widened on the way, by a load and a store.
template <class T>
__device__ __forceinline__ void stage_cell(C_t<T>* cell, const T* src, const TrapGrid& g, int gy,
                                           int gx, bool inside) {
  using C = C_t<T>;
  if constexpr (sizeof(T) == sizeof(C)) {
    if (!inside) {
      double v;
      if (outside_dirichlet(g, gy, gx, &v)) {
        *cell = C(v);
        return;
      }
      gy = wrap(gy, g.ny);
      gx = wrap(gx, g.nx);
    }
    cp_async_elem<sizeof(T)>(smem_u32(cell), src + int64_t(gy) * g.nx + gx);
  } else {
    *cell = inside ? to_c(__ldcg(src + int64_t(gy) * g.nx + gx)) : halo_read<T>(src, g, gy, gx);
  }
}

// One tile: k sweeps from src to dst.  smem holds 2 * NF * H * W values of C.
// Threads walk the window as a 2D grid (threadIdx.x along x in steps of 32,
// the rest of the block along y), so no cell index is divided.
template <class Op, class T>
__device__ __forceinline__ void trap_tile(const Op& op, const T* const* src, T* const* dst,
                                          const TrapGrid& g, int x0, int y0, int TX, int TY,
                                          int k, C_t<T>* smem) {
  using C = C_t<T>;
  constexpr int R = Op::R, NF = Op::NF;
  const int h = R * k;
  const int W = TX + 2 * h, H = TY + 2 * h, HW = W * H;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32, ny_t = blockDim.x / 32;
  C* b0 = smem;
  C* b1 = smem + NF * HW;
  // The whole window lies inside the grid: no boundary rule, no wrap.
  const bool inside = x0 - h >= 0 && y0 - h >= 0 && x0 + TX + h <= g.nx && y0 + TY + h <= g.ny;
  for (int j = ty; j < H; j += ny_t) {
    const int gy = y0 - h + j;
    for (int i = tx; i < W; i += 32) {
      const int gx = x0 - h + i;
#pragma unroll
      for (int f = 0; f < NF; ++f) stage_cell<T>(b0 + f * HW + j * W + i, src[f], g, gy, gx, inside);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int s = 1; s <= k; ++s) {
    const C* cur = (s & 1) ? b0 : b1;
    C* nxt = (s & 1) ? b1 : b0;
    const int lo = s * R;
    for (int j = lo + ty; j < H - lo; j += ny_t) {
      const int gy = y0 - h + j;
      for (int i = lo + tx; i < W - lo; i += 32) {
        const int gx = x0 - h + i;
        double v;
        if (!inside && outside_dirichlet(g, gy, gx, &v)) {
#pragma unroll
          for (int f = 0; f < NF; ++f) nxt[f * HW + j * W + i] = C(v);
          continue;
        }
        TrapAcc<C, NF> acc{cur, W, HW, i, j};
        C o[NF];
        C unused = C(0);
        op(acc, o, unused);
#pragma unroll
        for (int f = 0; f < NF; ++f) nxt[f * HW + j * W + i] = to_storage_precision<T>(o[f]);
      }
    }
    __syncthreads();
  }
  const C* fin = (k & 1) ? b1 : b0;
  for (int j = ty; j < TY; j += ny_t) {
    const int gy = y0 + j;
    if (gy >= g.ny) break;
    for (int i = tx; i < TX; i += 32) {
      const int gx = x0 + i;
      if (gx < g.nx) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
          dst[f][int64_t(gy) * g.nx + gx] = from_c<T>(fin[f * HW + (j + h) * W + (i + h)]);
      }
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ fixed shape
// The trapezoid tile with its shape (TX x TY, up to K sweeps) fixed at compile
// time, for 256-thread blocks: thread (tx, ty) = (lane, warp) owns the window
// cells (tx + 32c, ty + 8r), so every tap of the local function is a shared
// load at a compile-time offset from the cell's address.  Each sweep updates
// every cell of [R, W-R) x [R, H-R), a superset of the shrinking trapezoid
// region: a cell outside the region after sweep s is computed from values
// that are no longer exact, but it only feeds cells outside the region of
// sweep s+1, so the central TX x TY tile is exact after the last sweep (the
// same values the variable-shape trap_tile computes, operation for
// operation).  Windows that cross a Dirichlet side mask those cells to the
// halo value in every sweep; periodic windows need no mask (the window holds
// the periodic extension).
template <class C, int NF, int W, int HW>
struct FixedAcc {
  const C* p;  // the cell in field 0 of the current buffer
  __device__ __forceinline__ C operator()(int f, int dx, int dy, int) const {
    return p[f * HW + dy * W + dx];
  }
  __device__ __forceinline__ int64_t gidx() const { return 0; }
};

template <class Op, class T, int TX, int TY, int K>
struct TrapFixed {
  using C = C_t<T>;
  static constexpr int R = Op::R, NF = Op::NF;
  static constexpr int h = R * K, W = TX + 2 * h, H = TY + 2 * h, HW = W * H;
  static constexpr int NXC = (W + 31) / 32, NYC = (H + 7) / 8;
  static constexpr size_t SMEM = 2 * size_t(NF) * HW * sizeof(C);

  // kp <= K sweeps from src to dst for the tile at (x0, y0); blockDim.x = 256.
  static __device__ __forceinline__ void tile(const Op& op, const T* const* src, T* const* dst,
                                              const TrapGrid& g, int x0, int y0, int kp, C* smem) {
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    C* b0 = smem;
    C* b1 = smem + NF * HW;
    const bool inside = x0 - h >= 0 && y0 - h >= 0 && x0 + TX + h <= g.nx && y0 + TY + h <= g.ny;
    const bool dirichlet = g.bc[0][0] == kDirichlet || g.bc[0][1] == kDirichlet ||
                           g.bc[1][0] == kDirichlet || g.bc[1][1] == kDirichlet;
    const bool masked = !inside && dirichlet;
#pragma unroll
    for (int r = 0; r < NYC; ++r) {
      const int j = ty + 8 * r;
      if (j >= H) break;
      const int gy = y0 - h + j;
#pragma unroll
      for (int c = 0; c < NXC; ++c) {
        const int i = tx + 32 * c;
        if (i < W) {
          const int gx = x0 - h + i;
#pragma unroll
          for (int f = 0; f < NF; ++f)
            stage_cell<T>(b0 + f * HW + j * W + i, src[f], g, gy, gx, inside);
        }
      }
    }
    cp_async_wait_all();
    __syncthreads();
    for (int s = 1; s <= kp; ++s) {
      const C* cur = (s & 1) ? b0 : b1;
      C* nxt = (s & 1) ? b1 : b0;
#pragma unroll
      for (int r = 0; r < NYC; ++r) {
        const int j = ty + 8 * r;
        if (j < R || j >= H - R) continue;
#pragma unroll
        for (int c = 0; c < NXC; ++c) {
          const int i = tx + 32 * c;
          if (i < R || i >= W - R) continue;
          const int o = j * W + i;
          double v;
          if (masked && outside_dirichlet(g, y0 - h + j, x0 - h + i, &v)) {
#pragma unroll
            for (int f = 0; f < NF; ++f) nxt[f * HW + o] = C(v);
            continue;
          }
          FixedAcc<C, NF, W, HW> acc{cur + o};
          C out[NF];
          C unused = C(0);
          op(acc, out, unused);
#pragma unroll
          for (int f = 0; f < NF; ++f) nxt[f * HW + o] = to_storage_precision<T>(out[f]);
        }
      }
      __syncthreads();
    }
    const C* fin = (kp & 1) ? b1 : b0;
#pragma unroll
    for (int r = 0; r < NYC; ++r) {
      const int j = ty + 8 * r;
      if (j < h || j >= h + TY) continue;
      const int gy = y0 + j - h;
      if (gy >= g.ny) continue;
#pragma unroll
      for (int c = 0; c < NXC; ++c) {
        const int i = tx + 32 * c;
        if (i < h || i >= h + TX) continue;
        const int gx = x0 + i - h;
        if (gx < g.nx) {
#pragma unroll
          for (int f = 0; f < NF; ++f)
            dst[f][int64_t(gy) * g.nx + gx] = from_c<T>(fin[f * HW + j * W + i]);
        }
      }
    }
    __syncthreads();
  }
};

// One sweep of the window region [lo, W-lo) x [lo, H-lo) for the multi-stage
// tile: nxt = E(cur), or, when `comb`, nxt = a * base + b * E(cur) (base read
// at the local element only).  Cells outside a Dirichlet side keep their halo
// value.  Every value is rounded to the storage precision, as a stage written
// to memory would be.
template <class Op, class T>
__device__ __forceinline__ void trap_rk_sweep(const Op& op, const C_t<T>* cur, C_t<T>* nxt,
                                              const C_t<T>* base, bool comb, const Coef& ca,
                                              const Coef& cb, const TrapGrid& g, int x0, int y0,
                                              int h, int W, int H, int lo, bool inside) {
  using C = C_t<T>;
  constexpr int NF = Op::NF;
  const int HW = W * H;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32, ny_t = blockDim.x / 32;
  for (int j = lo + ty; j < H - lo; j += ny_t) {
    const int gy = y0 - h + j;
    for (int i = lo + tx; i < W - lo; i += 32) {
      const int gx = x0 - h + i;
      double v;
      if (!inside && outside_dirichlet(g, gy, gx, &v)) {
#pragma unroll
        for (int f = 0; f < NF; ++f) nxt[f * HW + j * W + i] = C(v);
        continue;
      }
      TrapAcc<C, NF> acc{cur, W, HW, i, j};
      C o[NF];
      C unused = C(0);
      op(acc, o, unused);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        C r = o[f];
        if (comb) r = fma_(cb.get(C()), r, mul(ca.get(C()), base[f * HW + j * W + i]));
        nxt[f * HW + j * W + i] = to_storage_precision<T>(r);
      }
    }
  }
  __syncthreads();
}

// Multi-stage (Runge-Kutta) steps fused in one tile: k steps of `stages`
// stages, each stage one sweep of the local function E plus, from stage 2 on,
// a pointwise combination with the state at the start of the step (the
// strong-stability-preserving forms of Shu and Osher, see rk_coeffs).  The
// window carries a halo of R * stages * k cells; each stage shrinks the valid
// region by R, exactly as k * stages plain sweeps would.  The intermediate
// stage states -- the storage the paper's Limitations paragraph (Sec. 5) says
// LOPe does not provide -- live in shared memory only.  smem holds 3 * NF * H
// * W values of C.
template <class Op, class T>
__device__ __forceinline__ void trap_tile_rk(const Op& op, const T* const* src, T* const* dst,
                                             const TrapGrid& g, int x0, int y0, int TX, int TY,
                                             int k, int stages, C_t<T>* smem) {
  using C = C_t<T>;
  constexpr int R = Op::R, NF = Op::NF;
  const int h = R * stages * k;
  const int W = TX + 2 * h, H = TY + 2 * h, HW = W * H;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32, ny_t = blockDim.x / 32;
  C* bu = smem;
  C* b1 = smem + NF * HW;
  C* b2 = smem + 2 * NF * HW;
  const bool inside = x0 - h >= 0 && y0 - h >= 0 && x0 + TX + h <= g.nx && y0 + TY + h <= g.ny;
  for (int j = ty; j < H; j += ny_t) {
    const int gy = y0 - h + j;
    for (int i = tx; i < W; i += 32) {
      const int gx = x0 - h + i;
#pragma unroll
      for (int f = 0; f < NF; ++f) stage_cell<T>(bu + f * HW + j * W + i, src[f], g, gy, gx, inside);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  Coef a2, b2c, a3, b3c;
  {
    double a, b;
    rk_coeffs(stages, 2, &a, &b);
    a2 = a;
    b2c = b;
    rk_coeffs(stages, 3, &a, &b);
    a3 = a;
    b3c = b;
  }
  int lo = 0;
  for (int step = 0; step < k; ++step) {
    lo += R;
    trap_rk_sweep<Op, T>(op, bu, b1, nullptr, false, a2, b2c, g, x0, y0, h, W, H, lo, inside);
    lo += R;
    trap_rk_sweep<Op, T>(op, b1, b2, bu, true, a2, b2c, g, x0, y0, h, W, H, lo, inside);
    if (stages == 2) {
      C* t = bu; bu = b2; b2 = t;
    } else {
      lo += R;
      trap_rk_sweep<Op, T>(op, b2, b1, bu, true, a3, b3c, g, x0, y0, h, W, H, lo, inside);
      C* t = bu; bu = b1; b1 = t;
    }
  }
  for (int j = ty; j < TY; j += ny_t) {
    const int gy = y0 + j;
    if (gy >= g.ny) break;
    for (int i = tx; i < TX; i += 32) {
      const int gx = x0 + i;
      if (gx < g.nx) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
          dst[f][int64_t(gy) * g.nx + gx] = from_c<T>(bu[f * HW + (j + h) * W + (i + h)]);
      }
    }
  }
  __syncthreads();
}

}  // namespace lope
