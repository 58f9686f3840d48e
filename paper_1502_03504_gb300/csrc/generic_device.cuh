// Kernels for any grid shape, alignment and stencil shape (device templates;
// compiles under nvcc and NVRTC alike):
//  * trap2d_kernel — shared-memory trapezoid tiles with temporal blocking
//    (2D; box stencils with corners allowed; see trap.cuh);
//  * trap2d_rk_kernel — the same tiles running fused Runge-Kutta steps;
//  * direct_kernel — one thread per output point reading its halo straight
//    from global memory through the boundary rule (2D and 3D).  This is the
//    plainest GPU form of "call the local function for each interior index"
//    (Sec. 2.2, Sec. 3.2) and serves shapes the TMA path cannot take;
//  * march3d_plain_kernel — 3D columns marched along z with the column in
//    registers, for grids the TMA tiles cannot stage.
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
// Taps of one output point.  A point whose whole halo box lies inside the
// grid reads at constant offsets from its own index; any other point applies
// the boundary rule per axis (a Dirichlet side gives its value; a periodic
// side wraps by one period, since the radius never exceeds a periodic extent).
template <class T, int NF>
struct GlobalAcc {
  using C = C_t<T>;
  const T* const* f;
  const Geom* g;
  int64_t p, plane;
  int z, y, x, nx;
  bool inside;
  __device__ __forceinline__ C operator()(int fi, int dx, int dy, int dz) const {
    if (inside) return to_c(__ldg(f[fi] + p + dz * plane + int64_t(dy) * nx + dx));
    int q[3] = {z + dz, y + dy, x + dx};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int n = int(g->n[ax]);
      if (q[ax] < 0) {
        if (g->bc[ax][0] == kDirichlet) return C(g->bval[ax][0]);
        q[ax] += n;
      } else if (q[ax] >= n) {
        if (g->bc[ax][1] == kDirichlet) return C(g->bval[ax][1]);
        q[ax] -= n;
      }
    }
    return to_c(__ldg(f[fi] + (int64_t(q[0]) * g->n[1] + q[1]) * nx + q[2]));
  }
  __device__ __forceinline__ int64_t gidx() const { return p; }
};

// The grid is cut into units of 256 consecutive points of one row (the last
// unit of a row may be short); block b takes a contiguous range of units and
// thread t the point t of each, so loads and stores are coalesced along x and
// the row and plane of each unit follow by counting, without a division per
// point.  (Evaluating four units per thread before storing, to keep more
// loads in flight, measured slower: 5.5 ms against 4.3 ms for 20 sweeps of a
// 7094^2 FP32 grid.)
template <class Op, class T>
__global__ void __launch_bounds__(256) direct_kernel(Op op, const __grid_constant__ Geom g,
                                                     const T* in0, const T* in1, const T* in2,
                                                     T* out0, T* out1, T* out2, double* partials) {
  using C = C_t<T>;
  constexpr int R = Op::R;
  const T* src[3] = {in0, in1, in2};
  T* dst[3] = {out0, out1, out2};
  const int nz = int(g.n[0]), ny = int(g.n[1]), nx = int(g.n[2]);
  const int chunks = (nx + 255) / 256;
  const int64_t units = int64_t(nz) * ny * chunks;
  const int64_t per = (units + gridDim.x - 1) / gridDim.x;
  int64_t u = int64_t(blockIdx.x) * per;
  const int64_t u1 = u + per < units ? u + per : units;
  double red = 0.0;
  if (u < u1) {
    const int64_t row = u / chunks;
    int c = int(u - row * chunks);
    int z = int(row / ny), y = int(row - int64_t(z) * ny);
    GlobalAcc<T, Op::NF> acc;
    acc.f = src;
    acc.g = &g;
    acc.plane = int64_t(nx) * ny;
    acc.nx = nx;
    for (; u < u1; ++u) {
      const int x = c * 256 + int(threadIdx.x);
      if (x < nx) {
        acc.z = z;
        acc.y = y;
        acc.x = x;
        acc.p = (int64_t(z) * ny + y) * nx + x;
        acc.inside = x >= R && x + R < nx && y >= R && y + R < ny &&
                     (g.ndim == 2 || (z >= R && z + R < nz));
        C o[Op::NF];
        C r1 = C(0);
        op(acc, o, r1);
        red += double(r1);
#pragma unroll
        for (int f = 0; f < Op::NF; ++f) dst[f][acc.p] = from_c<T>(o[f]);
      }
      if (++c == chunks) {
        c = 0;
        if (++y == ny) {
          y = 0;
          ++z;
        }
      }
    }
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

// ------------------------------------------------------------------ column march
// 3D sweeps for grids the TMA tiles cannot stage (a row pitch that is not a
// multiple of 16 bytes).  A 256-thread block owns a kMarchX x kMarchY tile of
// (x, y) columns and marches a chunk of planes [z0, z1).  Each thread keeps
// its column's values of planes z-R .. z+R in registers and loads the planes
// ahead of z PF steps early, so PF loads per field are in flight.  Taps off
// the column read the state at plane z+dz through the cache (the block's own
// columns, loaded one to R steps earlier, mostly hit L1); their addresses are
// sums of per-thread row offsets and per-step plane offsets held in
// registers.  The boundary rule is applied per axis from per-thread indexes:
// a wrapped index on a periodic axis, or a Dirichlet side (z checked first,
// then y, then x, as in the direct kernel), so every tap has the value the
// direct kernel reads.
constexpr int kMarchX = 32, kMarchY = 8;

template <class T, int NF, int R>
struct MarchAcc {
  using C = C_t<T>;
  const C (*q)[2 * R + 1];  // q[f][dz + R]: the column at plane z + dz
  const T* const* f;
  const Geom* g;
  const int* xi;  // wrapped x index per dx + R, or -1 / -2 past the low / high Dirichlet side
  const int* yi;
  const int* zi;
  const int64_t* yrow;  // yi * nx per dy + R
  const int64_t* zpl;   // zi * plane per dz + R (this step)
  int64_t p;
  __device__ __forceinline__ C side(int ax, int code) const {
    return C(g->bval[ax][code == -1 ? 0 : 1]);
  }
  __device__ __forceinline__ C operator()(int fi, int dx, int dy, int dz) const {
    if (dx == 0 && dy == 0) return q[fi][dz + R];
    const int zz = zi[dz + R], yy = yi[dy + R], xx = xi[dx + R];
    if (zz < 0) return side(0, zz);
    if (yy < 0) return side(1, yy);
    if (xx < 0) return side(2, xx);
    return to_c(__ldg(f[fi] + zpl[dz + R] + yrow[dy + R] + xx));
  }
  __device__ __forceinline__ int64_t gidx() const { return p; }
};

// Index of coordinate v on an axis of extent n: itself when inside, wrapped on
// a periodic side, or -1 / -2 past a low / high Dirichlet side.
__device__ __forceinline__ int axis_index(int v, int n, int bc_lo, int bc_hi) {
  if (v < 0) return bc_lo == kDirichlet ? -1 : v + n;
  if (v >= n) return bc_hi == kDirichlet ? -2 : v - n;
  return v;
}

template <class Op, class T>
__global__ void __launch_bounds__(256) march3d_plain_kernel(Op op, const __grid_constant__ Geom g,
                                                            const T* in0, const T* in1,
                                                            const T* in2, T* out0, T* out1,
                                                            T* out2, int zchunk) {
  using C = C_t<T>;
  constexpr int R = Op::R, NF = Op::NF, NQ = 2 * R + 1, PF = 4;
  const T* src[3] = {in0, in1, in2};
  T* dst[3] = {out0, out1, out2};
  const int nz = int(g.n[0]), ny = int(g.n[1]), nx = int(g.n[2]);
  const int tiles_x = (nx + kMarchX - 1) / kMarchX, tiles_y = (ny + kMarchY - 1) / kMarchY;
  const int tile = int(blockIdx.x % unsigned(tiles_x * tiles_y));
  const int chunk = int(blockIdx.x / unsigned(tiles_x * tiles_y));
  const int x = (tile % tiles_x) * kMarchX + int(threadIdx.x % kMarchX);
  const int y = (tile / tiles_x) * kMarchY + int(threadIdx.x / kMarchX);
  const int z0 = chunk * zchunk, z1 = min(nz, z0 + zchunk);
  if (x >= nx || y >= ny || z0 >= z1) return;
  const int64_t plane = int64_t(nx) * ny, col = int64_t(y) * nx + x;
  int xi[NQ], yi[NQ], zi[NQ];
  int64_t yrow[NQ], zpl[NQ];
#pragma unroll
  for (int d = 0; d < NQ; ++d) {
    xi[d] = axis_index(x + d - R, nx, g.bc[2][0], g.bc[2][1]);
    yi[d] = axis_index(y + d - R, ny, g.bc[1][0], g.bc[1][1]);
    yrow[d] = int64_t(yi[d]) * nx;
  }
  // The column's value at plane v (any v within R + PF of the chunk).
  auto column = [&](int f, int v) -> C {
    const int zz = axis_index(v, nz, g.bc[0][0], g.bc[0][1]);
    if (zz < 0) return C(g.bval[0][zz == -1 ? 0 : 1]);
    return to_c(__ldg(src[f] + zz * plane + col));
  };
  C q[NF][NQ], pend[NF][PF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
#pragma unroll
    for (int k = 0; k < NQ - 1; ++k) q[f][k] = column(f, z0 - R + k);
#pragma unroll
    for (int j = 0; j < PF; ++j) pend[f][j] = z0 + R + j < z1 + R ? column(f, z0 + R + j) : C(0);
  }
  MarchAcc<T, NF, R> acc;
  acc.q = q;
  acc.f = src;
  acc.g = &g;
  acc.xi = xi;
  acc.yi = yi;
  acc.zi = zi;
  acc.yrow = yrow;
  acc.zpl = zpl;
  for (int z = z0; z < z1; ++z) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      q[f][NQ - 1] = pend[f][0];
#pragma unroll
      for (int j = 0; j < PF - 1; ++j) pend[f][j] = pend[f][j + 1];
      const int v = z + R + PF;
      pend[f][PF - 1] = v < z1 + R ? column(f, v) : C(0);
    }
#pragma unroll
    for (int d = 0; d < NQ; ++d) {
      zi[d] = axis_index(z + d - R, nz, g.bc[0][0], g.bc[0][1]);
      zpl[d] = zi[d] * plane;
    }
    acc.p = z * plane + col;
    C o[NF];
    C r1 = C(0);
    op(acc, o, r1);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      dst[f][acc.p] = from_c<T>(o[f]);
#pragma unroll
      for (int k = 0; k < NQ - 1; ++k) q[f][k] = q[f][k + 1];
    }
  }
}

}  // namespace
}  // namespace lope
