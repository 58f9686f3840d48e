// Kernels for any grid shape, alignment and stencil shape (device templates;
// compiles under nvcc and NVRTC alike):
//  * trap2d_kernel — shared-memory trapezoid tiles with temporal blocking
//    (2D; box stencils with corners allowed; see trap.cuh);
//  * trap2d_rk_kernel — the same tiles running fused Runge-Kutta steps;
//  * direct_kernel — one thread per output point reading its halo straight
//    from global memory through the boundary rule (2D and 3D).  This is the
//    plainest GPU form of "call the local function for each interior index"
//    (Sec. 2.2, Sec. 3.2) and serves shapes the TMA path cannot take;
//  * march3d_plain_kernel / march3d_async_kernel — 3D planes marched along z
//    through a shared-memory ring, for grids the TMA tiles cannot stage.
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
// side wraps by one period, since the radius never exceeds a periodic extent;
// an external side reads the caller's planes beyond the grid).
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
        if (g->bc[ax][0] == kPeriodic) q[ax] += n;
      } else if (q[ax] >= n) {
        if (g->bc[ax][1] == kDirichlet) return C(g->bval[ax][1]);
        if (g->bc[ax][1] == kPeriodic) q[ax] -= n;
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

// ------------------------------------------------------------------ plane march
// 3D sweeps for grids the TMA tiles cannot stage (a row pitch that is not a
// multiple of 16 bytes).  A 256-thread block owns a kMarchX x kMarchY tile of
// (x, y) columns (one output per thread and plane) and marches a chunk of
// planes [z0, z1).  Each plane's (kMarchX + 2R) x (kMarchY + 2R) window, halo
// included, is staged in shared memory in compute precision, with the boundary
// rule already applied: a wrapped position on a periodic side, or the side's
// value past a Dirichlet side (z checked first, then y, then x, as in the
// direct kernel), so every tap reads the value the direct kernel reads.  A
// ring of 2R + 2 planes holds z-R .. z+R and the plane being written.  The
// loads of planes z+R+1 .. z+R+PF are kept in registers, issued PF steps
// before their plane enters the ring, so they are in flight while earlier
// planes compute.  PF = 1 measured fastest (diff7 FP32 130 x 500 x 510, 20
// steps: 2.72 ms; 2.85 ms with PF = 3).
constexpr int kMarchX = 64, kMarchY = 4;

template <class C, int NF, int W, int H, int NS, int R>
struct PlaneAcc {
  const C* ring;  // NS planes x NF fields x H x W
  int slot0;      // ring slot of plane z - R
  int o;          // window offset of this thread's output cell
  int64_t p;
  __device__ __forceinline__ C operator()(int f, int dx, int dy, int dz) const {
    int sl = slot0 + dz + R;
    sl = sl >= NS ? sl - NS : sl;
    return ring[(sl * NF + f) * (W * H) + o + dy * W + dx];
  }
  __device__ __forceinline__ int64_t gidx() const { return p; }
};

template <class Op, class T>
__global__ void __launch_bounds__(256) march3d_plain_kernel(Op op, const __grid_constant__ Geom g,
                                                            const T* in0, const T* in1,
                                                            const T* in2, T* out0, T* out1,
                                                            T* out2, int zchunk) {
  using C = C_t<T>;
  constexpr int R = Op::R, NF = Op::NF, W = kMarchX + 2 * R, H = kMarchY + 2 * R;
  constexpr int NS = 2 * R + 2, CELLS = W * H, PER = (CELLS + 255) / 256, PF = 1;
  static_assert(kMarchX * kMarchY == 256, "one output per thread and plane");
  static_assert(sizeof(C) * NS * NF * CELLS <= 48 * 1024, "plane ring exceeds static shared memory");
  __shared__ C ring[NS * NF * CELLS];
  const T* src[3] = {in0, in1, in2};
  T* dst[3] = {out0, out1, out2};
  const int nz = int(g.n[0]), ny = int(g.n[1]), nx = int(g.n[2]);
  const int tiles_x = (nx + kMarchX - 1) / kMarchX, tiles_y = (ny + kMarchY - 1) / kMarchY;
  const unsigned ntiles = unsigned(tiles_x) * unsigned(tiles_y);
  const int tile = int(blockIdx.x % ntiles), chunk = int(blockIdx.x / ntiles);
  const int x0 = (tile % tiles_x) * kMarchX, y0 = (tile / tiles_x) * kMarchY;
  const int z0 = chunk * zchunk, z1 = min(nz, z0 + zchunk);
  if (z0 >= z1) return;  // the whole block
  const int64_t plane = int64_t(nx) * ny;
  // This thread's window cells: the in-plane position of the source value, or
  // which Dirichlet side gives it (1, 2: y low / high; 3, 4: x low / high),
  // or -1 for a cell no output reads (past the tile's valid cells + R).
  const int xend = min(x0 + kMarchX, nx) + R, yend = min(y0 + kMarchY, ny) + R;
  int64_t cpos[PER];
  int ccode[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int e = int(threadIdx.x) + 256 * j;
    const int gy = y0 - R + e / W, gx = x0 - R + e % W;
    cpos[j] = 0;
    if (e >= CELLS || gx >= xend || gy >= yend) {
      ccode[j] = -1;
      continue;
    }
    const int yy = axis_index(gy, ny, g.bc[1][0], g.bc[1][1]);
    const int xx = axis_index(gx, nx, g.bc[2][0], g.bc[2][1]);
    if (yy < 0) ccode[j] = yy == -1 ? 1 : 2;
    else if (xx < 0) ccode[j] = xx == -1 ? 3 : 4;
    else {
      ccode[j] = 0;
      cpos[j] = int64_t(yy) * nx + xx;
    }
  }
  auto load_plane = [&](int v, C (&val)[NF][PER]) {
    const int zz = axis_index(v, nz, g.bc[0][0], g.bc[0][1]);
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int c = ccode[j];
        if (zz < 0) val[f][j] = C(g.bval[0][zz == -1 ? 0 : 1]);
        else if (c == 0) val[f][j] = to_c(__ldg(src[f] + zz * plane + cpos[j]));
        else if (c > 0) val[f][j] = C(g.bval[(c + 1) / 2][(c + 1) % 2]);
        else val[f][j] = C(0);
      }
  };
  auto slot = [&](int v) { return (v - z0 + R) % NS; };
  auto store_plane = [&](int v, const C (&val)[NF][PER]) {
    C* base = ring + slot(v) * NF * CELLS;
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int e = int(threadIdx.x) + 256 * j;
        if (e < CELLS) base[f * CELLS + e] = val[f][j];
      }
  };
  C pend[PF][NF][PER];
  for (int v = z0 - R; v < z0 + R; ++v) {
    load_plane(v, pend[0]);
    store_plane(v, pend[0]);
  }
#pragma unroll
  for (int k = 0; k < PF; ++k)
    if (z0 + k < z1) load_plane(z0 + R + k, pend[k]);
  const int tx = int(threadIdx.x) % kMarchX, ty = int(threadIdx.x) / kMarchX;
  const int x = x0 + tx, y = y0 + ty;
  const bool valid = x < nx && y < ny;
  PlaneAcc<C, NF, W, H, NS, R> acc;
  acc.ring = ring;
  acc.o = (ty + R) * W + tx + R;
  for (int z = z0; z < z1; ++z) {
    store_plane(z + R, pend[0]);
#pragma unroll
    for (int k = 0; k < PF - 1; ++k)
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int j = 0; j < PER; ++j) pend[k][f][j] = pend[k + 1][f][j];
    if (z + PF < z1) load_plane(z + R + PF, pend[PF - 1]);
    __syncthreads();
    if (valid) {
      acc.slot0 = slot(z - R);
      acc.p = (int64_t(z) * ny + y) * nx + x;
      C o[NF];
      C r1 = C(0);
      op(acc, o, r1);
#pragma unroll
      for (int f = 0; f < NF; ++f) dst[f][acc.p] = from_c<T>(o[f]);
    }
  }
}

// The plane march for FP32 and FP64 grids (stored type = compute type).  A
// 256-thread block owns a kAsyncX x kAsyncY tile of (x, y) columns; thread
// (tx, ty) computes the kAsyncRY consecutive rows ty * kAsyncRY + r of column
// tx, holding that column of the current plane (its halo rows included) in
// registers, so only the off-column taps read shared memory.  The window
// cells move by asynchronous element copies (cp.async) straight into their
// ring slot, PF planes ahead of the plane being computed, so a block keeps PF
// planes of loads in flight without holding them in registers; cells given by
// a Dirichlet side are stored directly.  One copy group per plane: before
// computing plane z a thread waits until its copies of planes up to z + R
// have landed (at most PF - 1 younger groups pending), then the block barrier
// makes every thread's copies and stores visible and frees the slot of plane
// z - R - 1, which is refilled with plane z + R + PF.  The ring holds
// 2R + 1 + PF planes.  Every tap reads what the direct kernel reads.
constexpr int kAsyncX = 64, kAsyncY = 16, kAsyncRY = 4;

// Planes in flight, and the ring's bytes (dynamic shared memory): up to four
// planes ahead within a 64 KB ring.
template <class C, int NF, int R>
__host__ __device__ constexpr int march_async_depth() {
  constexpr int slot = NF * (kAsyncX + 2 * R) * (kAsyncY + 2 * R) * int(sizeof(C));
  constexpr int fit = (64 * 1024) / slot - (2 * R + 1);
  return fit < 1 ? 1 : fit > 4 ? 4 : fit;
}
template <class C, int NF, int R>
__host__ __device__ constexpr int march_async_smem() {
  return (2 * R + 1 + march_async_depth<C, NF, R>()) * NF * (kAsyncX + 2 * R) *
         (kAsyncY + 2 * R) * int(sizeof(C));
}

template <class C, int NF, int W, int CELLS, int R, int RY>
struct MarchColAcc {
  const C* pl[2 * R + 1];             // plane z + dz, at this thread's first output cell
  const C (*col)[NF][RY + 2 * R];     // plane z, this column, rows -R .. RY - 1 + R
  int r;                              // output row within the thread's rows
  int64_t p;                          // global index of the output
  __device__ __forceinline__ C operator()(int f, int dx, int dy, int dz) const {
    if (dx == 0 && dz == 0) return (*col)[f][r + R + dy];
    return pl[dz + R][f * CELLS + (r + dy) * W + dx];
  }
  __device__ __forceinline__ int64_t gidx() const { return p; }
};

template <class Op, class T>
__global__ void __launch_bounds__(256) march3d_async_kernel(Op op, const __grid_constant__ Geom g,
                                                            const T* in0, const T* in1,
                                                            const T* in2, T* out0, T* out1,
                                                            T* out2, int zchunk) {
  using C = C_t<T>;
  static_assert(sizeof(C) == sizeof(T), "stored type copied as is");
  constexpr int R = Op::R, NF = Op::NF, RY = kAsyncRY;
  constexpr int W = kAsyncX + 2 * R, H = kAsyncY + 2 * R, CELLS = W * H;
  constexpr int PER = (CELLS + 255) / 256;
  constexpr int PF = march_async_depth<C, NF, R>(), NS = 2 * R + 1 + PF;
  static_assert(kAsyncX * kAsyncY == 256 * RY, "RY outputs per thread and plane");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* const ring = reinterpret_cast<C*>(smem_raw);  // NS planes x NF fields x CELLS
  const T* src[3] = {in0, in1, in2};
  T* dst[3] = {out0, out1, out2};
  const int nz = int(g.n[0]), ny = int(g.n[1]), nx = int(g.n[2]);
  const int tiles_x = (nx + kAsyncX - 1) / kAsyncX, tiles_y = (ny + kAsyncY - 1) / kAsyncY;
  const unsigned ntiles = unsigned(tiles_x) * unsigned(tiles_y);
  const int tile = int(blockIdx.x % ntiles), chunk = int(blockIdx.x / ntiles);
  const int x0 = (tile % tiles_x) * kAsyncX, y0 = (tile / tiles_x) * kAsyncY;
  const int z0 = chunk * zchunk, z1 = min(nz, z0 + zchunk);
  if (z0 >= z1) return;  // the whole block
  const int64_t plane = int64_t(nx) * ny;
  // This thread's window cells: the in-plane position of the source value, or
  // which Dirichlet side gives it (1, 2: y low / high; 3, 4: x low / high),
  // or -1 for a cell no output reads (past the tile's valid cells + R).
  const int xend = min(x0 + kAsyncX, nx) + R, yend = min(y0 + kAsyncY, ny) + R;
  int64_t cpos[PER];
  int ccode[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int e = int(threadIdx.x) + 256 * j;
    const int gy = y0 - R + e / W, gx = x0 - R + e % W;
    cpos[j] = 0;
    if (e >= CELLS || gx >= xend || gy >= yend) {
      ccode[j] = -1;
      continue;
    }
    const int yy = axis_index(gy, ny, g.bc[1][0], g.bc[1][1]);
    const int xx = axis_index(gx, nx, g.bc[2][0], g.bc[2][1]);
    if (yy < 0) ccode[j] = yy == -1 ? 1 : 2;
    else if (xx < 0) ccode[j] = xx == -1 ? 3 : 4;
    else {
      ccode[j] = 0;
      cpos[j] = int64_t(yy) * nx + xx;
    }
  }
  const uint32_t sring = smem_u32(ring);
  auto slot = [&](int v) { return (v - z0 + R) % NS; };
  // Issue plane v into its slot and close its copy group (empty past the chunk).
  auto issue = [&](int v) {
    if (v < z1 + R) {
      const int zz = axis_index(v, nz, g.bc[0][0], g.bc[0][1]);
      const int base = slot(v) * NF * CELLS + int(threadIdx.x);
      const T* s0 = src[0] + (zz < 0 ? 0 : int64_t(zz) * plane);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const T* sf = f == 0 ? s0 : src[f] + (zz < 0 ? 0 : int64_t(zz) * plane);
#pragma unroll
        for (int j = 0; j < PER; ++j) {
          const int c = ccode[j];
          if (c < 0) continue;
          const int e = base + f * CELLS + 256 * j;
          if (zz < 0) ring[e] = C(g.bval[0][zz == -1 ? 0 : 1]);
          else if (c == 0)
            cp_async_elem<int(sizeof(T))>(sring + unsigned(e) * unsigned(sizeof(C)), sf + cpos[j]);
          else ring[e] = C(g.bval[(c + 1) / 2][(c + 1) % 2]);
        }
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  for (int v = z0 - R; v < z0 + R + PF; ++v) issue(v);
  const int tx = int(threadIdx.x) % kAsyncX, ty = int(threadIdx.x) / kAsyncX;
  const int x = x0 + tx, yb = y0 + ty * RY;
  const int cell0 = (ty * RY + R) * W + tx + R;  // window offset of the first output
  MarchColAcc<C, NF, W, CELLS, R, RY> acc;
  C col[NF][RY + 2 * R];
  acc.col = &col;
  for (int z = z0; z < z1; ++z) {
    asm volatile("cp.async.wait_group %0;" ::"n"(PF - 1) : "memory");
    __syncthreads();
    issue(z + R + PF);
    if (x < nx && yb < ny) {
      int sl = slot(z - R);
#pragma unroll
      for (int d = 0; d < 2 * R + 1; ++d) {
        acc.pl[d] = ring + sl * NF * CELLS + cell0;
        sl = sl + 1 == NS ? 0 : sl + 1;
      }
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int k = 0; k < RY + 2 * R; ++k) col[f][k] = acc.pl[R][f * CELLS + (k - R) * W];
      const int64_t p0 = (int64_t(z) * ny + yb) * nx + x;
      auto row = [&](int r) {
        acc.r = r;
        acc.p = p0 + int64_t(r) * nx;
        C o[NF];
        C r1 = C(0);
        op(acc, o, r1);
#pragma unroll
        for (int f = 0; f < NF; ++f) dst[f][acc.p] = from_c<T>(o[f]);
      };
      if constexpr (Op::STAR || R == 1) {
#pragma unroll
        for (int r = 0; r < RY; ++r)
          if (yb + r < ny) row(r);
      } else {  // 125-tap boxes: one row at a time keeps the weights in registers
#pragma unroll 1
        for (int r = 0; r < RY; ++r)
          if (yb + r < ny) row(r);
      }
    }
  }
  cp_async_wait_all();
}

}  // namespace
}  // namespace lope
