// TMA-staged stencil kernels (device templates).  Included by tma_kernels.cuh
// (the host-side runner) and, as embedded source, by run-time compiled local
// functions (jit.cu); it compiles under nvcc and NVRTC alike.
//
// The paper's multi-level halo exchange (Sec. 3.2 HALO_TRANSFER; Sec. 3.3 on
// halo elements being several memory hops away) becomes, on one GB300, the
// HBM -> shared memory -> register hierarchy:
//   * a producer warp stages halo-padded tiles into a ring of shared-memory
//     stages with cp.async.bulk.tensor (TMA), one mbarrier per stage;
//   * ghost cells are produced by the copy itself: out-of-range boxes are
//     zero-filled by the TMA unit (Dirichlet 0) and periodic halos are fetched
//     from wrapped coordinates (BC=CYCLIC, Sec. 3.2);
//   * consumer threads run the local function, one thread per output column,
//     RY rows each; in 3D each thread marches along z keeping the 2R+1 centre
//     values of its column in a register queue.
//
// Shared-memory stage layout for one field (TX x TY tile, radius R):
//   main  (TY + 2R) rows x TX     rows y0-R .. y0+TY+R-1 (low halo, body, high halo)
//   left  TY rows x CW            columns x0-CW .. x0-1     (CW = 16 bytes of elements)
//   right TY rows x CW            columns x0+nvx .. x0+nvx+CW-1
// Star stencils never read corners, so the slots only span the body rows.
// When the high halo of a ragged or periodic tile does not follow the body in
// memory, it is fetched separately into the rows after TY; the accessor maps
// row >= nvy there.
//
// Box stencils (corner taps, 2D only) take no slots: the wide box already
// holds the corners of interior tiles, and on tiles whose halo wraps the
// consumer warps rewrite the halo ring of the box from the wrapped global
// coordinates before reading it (fill_ring_warp).
#pragma once

#include "device_common.cuh"

namespace lope {

namespace {

// Tile shape per storage type, rank and field count: TX columns (TX times the
// element size is a multiple of 128 bytes), TY rows, RY rows per consumer
// thread (TX * TY / RY consumer threads plus one producer warp), S stages.
template <class T> struct TmaTx { static constexpr int TX = 64; };
template <> struct TmaTx<double> { static constexpr int TX = 32; };

//
// Single-field paired kernels take tall tiles: 128 rows in 2D (the 2R halo
// rows that neighbouring tiles read again are 2R/128 of a tile; the 3-stage
// ring of 17-warp blocks holds one block per SM) and 64 rows in 3D; measured
// on GB300 against shorter tiles and other depths (2D 9-point 8192^2: 0.74 ->
// 0.91 of the copy peak; 3D 7-point 512^3: 0.905 -> 0.926; radius-1 only in
// 3D, where a radius-2 register queue of 8 rows would spill).  FP32
// multi-field 2D tiles are 64 rows with 4 rows per thread (17-warp blocks:
// nonlinear shallow water 0.44 -> 0.53, Gray-Scott 0.75 -> 0.86; the linear
// shallow water unchanged).  Three-field 3D rings take 6 stages (5 at radius
// 2) to stay within 227 KB of shared memory.
// TALL = false gives the shorter tiles (2D single-field 64 rows, others 32),
// which keep more blocks in flight on small grids; the runner picks per grid.
template <class T, int RANK, int R, int NF, bool PAIR, bool TALL = true> struct TmaCfg {
  static constexpr int TX = TmaTx<T>::TX;
  static constexpr bool TALL2 = TALL && RANK == 2 && NF == 1 && PAIR;
  static constexpr bool TALL3 = TALL && RANK == 3 && NF == 1 && PAIR && R == 1;
  static constexpr bool MULTI = TALL && RANK == 2 && NF > 1 && PAIR;
  static constexpr int TY = TALL2 ? 128 : (RANK == 2 && NF == 1) ? 64 : (TALL3 || MULTI) ? 64 : 32;
  static constexpr int RY = PAIR ? (((RANK == 2 && NF == 1) || TALL3) ? 8 : 4) : (RANK == 2 ? 16 : 8);
  static constexpr int S = RANK == 3 ? (NF == 3 ? (R == 2 ? 5 : 6) : 8) : 3;
};

template <int NF> struct TmaMaps {
  CUtensorMap wide[NF];  // box {W, TY+2R}: tile, CW halo columns each side, R halo rows each side
  CUtensorMap rows[NF];  // box {W, R}: R consecutive halo rows
  CUtensorMap cols[NF];  // box {CW, TY} (star functions: the body rows) or {CW, TY+2R} (box
                         // functions: the halo rows too): one 16-byte column block
};

template <class Op, class T> struct TmaParams {
  Op op;
  const T* in[kMaxFields];  // the staged fields (read directly only by fill_ring_warp)
  T* out[kMaxFields];
  int nx, ny, nz;
  int per_x, per_y, per_z;
  int tiles_x, tiles_y;
  int zchunk;     // 3D: output planes per unit
  int nunits;     // number of work units
  int soff;       // slowest-axis planes (3D) / rows (2D) the tensor maps hold
                  // before the grid: the external halo of a slab (else 0)
  int sext;       // external sides of the slowest axis: bit 0 low, bit 1 high
  double* partials;
  int* err;
};

// Stage layout (per field, every region 128-byte aligned, as TMA requires):
//   wide   (TY+2R) x W box, W = TX + 2 CW, loaded at (x0-CW, y0-R): the tile,
//          CW halo columns on each side and R halo rows above and below.
//          Out-of-range cells arrive as zeros (the Dirichlet-0 halo).
//   colL, colR   (TY+2R) x CW slots: wrapped halo columns (periodic x edge
//                tiles; TY rows for star functions, TY+2R for box functions)
//   rowLo, rowHi R x W slots: wrapped halo rows (periodic y edge tiles)
// Consumers read every tap at a compile-time offset from the local element in
// the wide box.  Where the periodic halo wraps (BC=CYCLIC of Sec. 3.2), the
// wrapped halo rows feed the column registers from the row slots, and the
// warps that read the wrapped halo columns first copy them from the column
// slots into the box.  Star stencils never read the corner cells.
template <class T, int TX, int TY, int R, int NF> struct Layout {
  static constexpr int CW = 16 / int(sizeof(T));
  static constexpr int W = TX + 2 * CW;
  static constexpr uint32_t WIDE_B = (TY + 2 * R) * W * sizeof(T);
  static constexpr uint32_t COL_B = TY * CW * sizeof(T);             // star functions
  static constexpr uint32_t COLX_B = (TY + 2 * R) * CW * sizeof(T);  // box functions
  static constexpr uint32_t ROW_B = R * W * sizeof(T);
  static constexpr uint32_t A(uint32_t b) { return (b + 127) / 128 * 128; }
  static constexpr uint32_t OFF_COLL = A(WIDE_B);
  static constexpr uint32_t OFF_COLR = OFF_COLL + A(COLX_B);
  static constexpr uint32_t OFF_ROWLO = OFF_COLR + A(COLX_B);
  static constexpr uint32_t OFF_ROWHI = OFF_ROWLO + A(ROW_B);
  static constexpr uint32_t FIELD_B = OFF_ROWHI + A(ROW_B);
  static constexpr uint32_t STAGE_B = NF * FIELD_B;
};

// Which halos of a tile wrap (periodic axes only).
struct TileInfo {
  int x0, y0, nvx, nvy;
  bool xl, xr;  // left / right halo columns wrap
  bool yl, yh;  // low / high halo rows wrap
};

template <class T, int TX, int TY, int R>
__device__ __forceinline__ TileInfo classify(int x0, int y0, int nx, int ny, int per_x, int per_y) {
  TileInfo t;
  t.x0 = x0;
  t.y0 = y0;
  t.nvx = min(TX, nx - x0);
  t.nvy = min(TY, ny - y0);
  t.xl = per_x && x0 == 0;
  t.xr = per_x && x0 + t.nvx == nx;
  t.yl = per_y && y0 < R;
  t.yh = per_y && y0 + t.nvy + R > ny;
  return t;
}

// Local-function accessor: x taps are shared loads at compile-time offsets
// from b[f] (the local element in the wide box); y taps and the centre come
// from the thread's column registers col[f][R + dy]; z taps (3D) from the
// register queue q[f][R + dz].
template <class T, int TX, int TY, int R, int NF, int NQ, int NC>
struct StageAcc {
  using C = C_t<T>;
  const T* b[NF];
  const C (*col)[NC];  // col[f] + r, so col[f][R + dy] is row r + dy
  int r;
  int64_t g;
  const C (*q)[NQ];
  __device__ __forceinline__ C operator()(int f, int dx, int dy, int dz) const {
    if (dz != 0) return q[f][R + dz];
    if (dx != 0) return to_c(b[f][dy * Layout<T, TX, TY, R, NF>::W + dx]);  // dy != 0: box corner
    return col[f][r + R + dy];
  }
  __device__ __forceinline__ int64_t gidx() const { return g; }
};

// Periodic x edge: copy the wrapped halo columns that this warp's own lanes
// will read (rows cy0 .. cy0+RY-1) from the column slots into the wide box.
// Left-halo readers (cx < R) and right-halo readers (nvx-R <= cx < nvx) each
// sit in a single warp, so a warp-level barrier is enough; the proxy fence
// orders these shared-memory writes before the stage's next TMA refill.
template <class T, int TX, int TY, int R, int NF, int RY>
__device__ __forceinline__ void fix_x_warp(unsigned char* st, const TileInfo& t, int cx, int cy0) {
  using L = Layout<T, TX, TY, R, NF>;
  const int lane = threadIdx.x % 32, cxw = cx - lane;  // first column of this warp
  const bool left = t.xl && cxw == 0;
  const bool right = t.xr && cxw <= t.nvx - 1 && t.nvx - 1 < cxw + 32;
  if (!left && !right) return;
  if (lane < R * RY) {
    const int d = lane / RY, r = lane % RY;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T* w = reinterpret_cast<T*>(st + f * L::FIELD_B);
      const T* sl = reinterpret_cast<const T*>(st + f * L::FIELD_B + L::OFF_COLL);
      const T* sr = reinterpret_cast<const T*>(st + f * L::FIELD_B + L::OFF_COLR);
      if (left) w[(R + cy0 + r) * L::W + L::CW - 1 - d] = sl[(cy0 + r) * L::CW + L::CW - 1 - d];
      if (right) w[(R + cy0 + r) * L::W + L::CW + t.nvx + d] = sr[(cy0 + r) * L::CW + d];
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
}

// Value for the column registers: tile row tr (which may lie in the halo) of
// column cx, taken from the wide box or, where the periodic halo wraps, from
// the wrapped row slots.
template <class T, int TX, int TY, int R, int NF>
__device__ __forceinline__ C_t<T> column_value(const unsigned char* st, int f, const TileInfo& t,
                                               int tr, int cx, int ny, bool yw) {
  using L = Layout<T, TX, TY, R, NF>;
  const unsigned char* fb = st + f * L::FIELD_B;
  if (yw) {
    if (t.yl && tr < 0)  // the low slot holds rows ny-R .. ny-1; y0 = 0 here
      return to_c(reinterpret_cast<const T*>(fb + L::OFF_ROWLO)[(tr + R) * L::W + L::CW + cx]);
    const int gy = t.y0 + tr;
    // The high slot holds rows 0 .. R-1.  Rows further out are read only for
    // rows below the grid edge, whose results are discarded: clamp in range.
    if (t.yh && gy >= ny)
      return to_c(reinterpret_cast<const T*>(fb + L::OFF_ROWHI)[min(gy - ny, R - 1) * L::W + L::CW + cx]);
  }
  return to_c(reinterpret_cast<const T*>(fb)[(R + tr) * L::W + L::CW + cx]);
}

template <int RANK>
__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* m, int x, int y, int z,
                                         uint64_t* bar) {
  if (RANK == 2) tma_load_2d(dst, m, x, y, bar);
  else tma_load_3d(dst, m, x, y, z, bar);
}

// Box functions on a tile whose halo wraps on one axis only take the wrapped
// halo from slots (fill_ring_slots); tiles at a corner of the grid, where it
// wraps on both axes, read the wrapped cells from global memory instead
// (fill_ring_warp).
__device__ __forceinline__ bool box_corner(const TileInfo& t) {
  return (t.xl || t.xr) && (t.yl || t.yh);
}

// What a stage holds besides the wide box (issue_plane's MODE).
enum : int {
  kStageStar = 0,  // star functions: wrapped halo columns (body rows) and rows in slots
  kStageBox = 1,   // box functions: wrapped halo columns (halo rows too) and rows in slots,
                   // none on corner tiles of the grid
  kStageWide = 2   // the wide box alone (the two-sweep kernels)
};

// Issue the copies of one tile/plane of every field into stage `st`.
// yoff: rows the 2D tensor maps hold before the grid (an external y halo).
template <class T, int TX, int TY, int R, int NF, int RANK, int MODE = kStageStar>
__device__ __forceinline__ void issue_plane(const TmaMaps<NF>& maps, unsigned char* st,
                                            uint64_t* bar, const TileInfo& t, int z, int nx,
                                            int ny, int yoff = 0) {
  using L = Layout<T, TX, TY, R, NF>;
  constexpr bool BOX = MODE == kStageBox;
  const bool slots = MODE == kStageStar || (BOX && !box_corner(t));
  const uint32_t per_field =
      L::WIDE_B + (slots ? (uint32_t(t.xl) + uint32_t(t.xr)) * (BOX ? L::COLX_B : L::COL_B) +
                               (uint32_t(t.yl) + uint32_t(t.yh)) * L::ROW_B
                         : 0u);
  mbar_arrive_expect_tx(bar, NF * per_field);
  const int xw = t.x0 - L::CW;
  const int cy = t.y0 + yoff - (BOX ? R : 0);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    unsigned char* w = st + f * L::FIELD_B;
    tma_load<RANK>(w, &maps.wide[f], xw, t.y0 - R + yoff, z, bar);
    if (!slots) continue;
    if (t.xl) tma_load<RANK>(w + L::OFF_COLL, &maps.cols[f], nx - L::CW, cy, z, bar);
    if (t.xr) tma_load<RANK>(w + L::OFF_COLR, &maps.cols[f], 0, cy, z, bar);
    if (t.yl) tma_load<RANK>(w + L::OFF_ROWLO, &maps.rows[f], xw, ny - R, z, bar);
    if (t.yh) tma_load<RANK>(w + L::OFF_ROWHI, &maps.rows[f], xw, 0, z, bar);
  }
}

// Round a shared-memory pointer up to 128 bytes.  The offset is added to the
// pointer itself (no round trip through an integer), so the compiler still
// knows every pointer derived from it addresses shared memory and emits
// shared loads and stores with 32-bit addresses.
__device__ __forceinline__ unsigned char* align128(unsigned char* p) {
  return p + ((128u - (smem_u32(p) & 127u)) & 127u);
}

// Sum an FP64 value over the consumer threads (named barrier 1) and add it to
// this block's partial slot.  Fixed order: deterministic.
template <int NCONS>
__device__ __forceinline__ void block_accumulate(double v, double* partials, double* scratch) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) scratch[warp] = v;
  asm volatile("bar.sync 1, %0;" ::"r"(NCONS) : "memory");
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NCONS / 32; ++w) s += scratch[w];
    partials[blockIdx.x] += s;
  }
}

// RY outputs of one column of a staged tile/plane.  col[f][i] holds the
// column's values for tile rows cy0 - R + i, i in [0, RY + 2R).
template <class Op, class T, int TX, int TY, int RY, int NQ, int NC>
__device__ __forceinline__ void column_rows(const Op& op, const unsigned char* st, T* const* out,
                                            int64_t zoff, int nx, const TileInfo& t, int cx,
                                            int cy0, const C_t<T> (*col)[NC],
                                            const C_t<T> (*q)[Op::NF][NQ], double& red) {
  using C = C_t<T>;
  constexpr int R = Op::R, NF = Op::NF;
  using L = Layout<T, TX, TY, R, NF>;
  const bool xvalid = cx < t.nvx;
  const int64_t base = zoff + int64_t(t.y0 + cy0) * nx + t.x0 + cx;
  const int64_t gclamp = zoff + int64_t(t.y0) * nx + t.x0;  // a valid element for clamped reads
  C rsum = C(0);  // adjoint terms of this column, summed in compute precision
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const bool valid = xvalid && cy0 + r < t.nvy;
    StageAcc<T, TX, TY, R, NF, NQ, NC> acc;
#pragma unroll
    for (int f = 0; f < NF; ++f)
      acc.b[f] = reinterpret_cast<const T*>(st + f * L::FIELD_B) + (R + cy0 + r) * L::W + L::CW + cx;
    acc.col = col;
    acc.r = r;
    acc.g = valid ? base + int64_t(r) * nx : gclamp;
    acc.q = q ? q[r] : nullptr;
    C o[NF];
    C r1 = C(0);
    op(acc, o, r1);
    if (valid) {
#pragma unroll
      for (int f = 0; f < NF; ++f) out[f][base + int64_t(r) * nx] = from_c<T>(o[f]);
      rsum = add(rsum, r1);
    }
  }
  if (Op::REDUCES) red += double(rsum);
}

// The R column values above (lo) and below (hi) a thread's strip of RY rows.
// `simple` (decided once per tile): the tile is not ragged in y and its high
// halo, if it wraps, wraps whole; then only row group 0 reads the low row slot
// and only the last row group the high one, a warp-uniform choice.  Other
// wrapped tiles take column_value for each row.
template <class T, int TX, int TY, int R, int NF, int RY, bool YW>
__device__ __forceinline__ void edge_rows(const unsigned char* st, int f, const TileInfo& t, int cx,
                                          int cy0, int ny, bool simple, C_t<T>* lo, C_t<T>* hi) {
  using L = Layout<T, TX, TY, R, NF>;
  const unsigned char* fb = st + f * L::FIELD_B;
  const T* box = reinterpret_cast<const T*>(fb);
  if (!YW) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      lo[k] = to_c(box[(cy0 + k) * L::W + L::CW + cx]);
      hi[k] = to_c(box[(cy0 + R + RY + k) * L::W + L::CW + cx]);
    }
  } else if (simple) {
    const T* lsrc = (t.yl && cy0 == 0) ? reinterpret_cast<const T*>(fb + L::OFF_ROWLO)
                                       : box + cy0 * L::W;
    const T* hsrc = (t.yh && cy0 + RY == TY) ? reinterpret_cast<const T*>(fb + L::OFF_ROWHI)
                                             : box + (cy0 + R + RY) * L::W;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      lo[k] = to_c(lsrc[k * L::W + L::CW + cx]);
      hi[k] = to_c(hsrc[k * L::W + L::CW + cx]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      lo[k] = column_value<T, TX, TY, R, NF>(st, f, t, cy0 - R + k, cx, ny, true);
      hi[k] = column_value<T, TX, TY, R, NF>(st, f, t, cy0 + RY + k, cx, ny, true);
    }
  }
}

template <int TY>
__device__ __forceinline__ bool simple_y(const TileInfo& t, int ny) {
  return t.nvy == TY && (!t.yh || t.y0 + TY == ny);
}

// One staged 2D tile: wrapped x halo patched by the warps that read it,
// column registers (wrapped halo rows from the row slots when YW), then rows.
template <bool YW, bool SIMPLE, bool WRAP, class Op, class T, int TX, int TY, int RY>
__device__ __forceinline__ void tile2d(const Op& op, unsigned char* st, T* const* out, int nx,
                                       int ny, const TileInfo& t, int cx, int cy0, double& red) {
  using C = C_t<T>;
  constexpr int R = Op::R, NF = Op::NF, NC = RY + 2 * R;
  using L = Layout<T, TX, TY, R, NF>;
  if (WRAP && (t.xl || t.xr)) fix_x_warp<T, TX, TY, R, NF, RY>(st, t, cx, cy0);
  constexpr bool simple = !YW || SIMPLE;
  C col[NF][NC];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    edge_rows<T, TX, TY, R, NF, RY, YW>(st, f, t, cx, cy0, ny, simple, &col[f][0], &col[f][R + RY]);
    const T* box = reinterpret_cast<const T*>(st + f * L::FIELD_B);
    if (simple) {
#pragma unroll
      for (int r = 0; r < RY; ++r) col[f][R + r] = to_c(box[(R + cy0 + r) * L::W + L::CW + cx]);
    } else {
#pragma unroll
      for (int r = 0; r < RY; ++r)
        col[f][R + r] = column_value<T, TX, TY, R, NF>(st, f, t, cy0 + r, cx, ny, true);
    }
  }
  column_rows<Op, T, TX, TY, RY, 1, NC>(op, st, out, 0, nx, t, cx, cy0, col, nullptr, red);
}

// ------------------------------------------------------------------ column pairs
// Paired consumers (FP32/BF16 storage): each thread computes two adjacent
// columns cx2, cx2+1 with the packed f32x2 instructions (adjoint functors'
// per-point terms are summed per lane and added to the FP64 block sum).  Pair loads and
// stores are 8 bytes (FP32) or 4 bytes (BF16) and aligned, since cx2, CW and
// the box width are even.  x taps of radius <= 2 come from the aligned pairs
// left (cx2-2, cx2-1) and right (cx2+2, cx2+3) of the centre pair.
__device__ __forceinline__ F2 ld_pair(const float* p) {
  F2 r;
  r.v = *reinterpret_cast<const uint64_t*>(p);
  return r;
}
// A BF16 value is the upper half of the FP32 value it widens to, so a pair
// widens exactly with one shift (low element) and one mask (high element).
__device__ __forceinline__ F2 ld_pair(const __nv_bfloat16* p) {
  const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
  return F2::make(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
// One element of an aligned pair: p[0] (lo) or p[1] (hi); a BF16 element
// widens from the pair's word with one instruction.
__device__ __forceinline__ float ld_pair_lo(const float* p) { return ld_pair(p).lo(); }
__device__ __forceinline__ float ld_pair_hi(const float* p) { return ld_pair(p).hi(); }
__device__ __forceinline__ float ld_pair_lo(const __nv_bfloat16* p) {
  return __uint_as_float(*reinterpret_cast<const uint32_t*>(p) << 16);
}
__device__ __forceinline__ float ld_pair_hi(const __nv_bfloat16* p) {
  return __uint_as_float(*reinterpret_cast<const uint32_t*>(p) & 0xffff0000u);
}
__device__ __forceinline__ void st_pair(float* p, F2 v) { *reinterpret_cast<uint64_t*>(p) = v.v; }
// Both elements rounded to nearest even and packed by one conversion.
__device__ __forceinline__ void st_pair(__nv_bfloat16* p, F2 v) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.lo(), v.hi());
}

template <class T, int TX, int TY, int R, int NF, int NC>
struct PairAcc {
  static_assert(R <= 2, "paired taps reach two columns");
  const T* b[NF];      // centre pair of this row in the wide box
  const F2 (*col)[NC];
  int r;
  int64_t g;
  __device__ __forceinline__ F2 operator()(int f, int dx, int dy, int) const {
    if (dx == 0) return col[f][r + R + dy];
    const T* rb = b[f] + dy * Layout<T, TX, TY, R, NF>::W;  // row r + dy (corner taps of box stencils)
    if (dx == -2) return ld_pair(rb - 2);
    if (dx == 2) return ld_pair(rb + 2);
    const F2 c = col[f][r + R + dy];
    if (dx == -1) return F2::make(ld_pair_hi(rb - 2), c.lo());
    return F2::make(c.hi(), ld_pair_lo(rb + 2));
  }
  __device__ __forceinline__ int64_t gidx() const { return g; }
};

// 3D variant: z taps come from the register queue of packed pairs.
template <class T, int TX, int TY, int R, int NF, int NC, int NQ>
struct PairAcc3 {
  const T* b[NF];
  const F2 (*col)[NC];
  int r;
  int64_t g;
  const F2 (*q)[NQ];
  __device__ __forceinline__ F2 operator()(int f, int dx, int dy, int dz) const {
    if (dz != 0) return q[f][R + dz];
    if (dx == 0) return col[f][r + R + dy];
    if (dx == -2) return ld_pair(b[f] - 2);
    if (dx == 2) return ld_pair(b[f] + 2);
    const F2 c = col[f][r + R];
    if (dx == -1) return F2::make(ld_pair_hi(b[f] - 2), c.lo());
    return F2::make(c.hi(), ld_pair_lo(b[f] + 2));
  }
  __device__ __forceinline__ int64_t gidx() const { return g; }
};

// Pair value of tile row tr for the column registers: from the wide box or,
// where the periodic y halo wraps, from the row slots (as column_value).
template <class T, int TX, int TY, int R, int NF>
__device__ __forceinline__ F2 column_pair(const unsigned char* st, int f, const TileInfo& t, int tr,
                                          int cx2, int ny) {
  using L = Layout<T, TX, TY, R, NF>;
  const unsigned char* fb = st + f * L::FIELD_B;
  if (t.yl && tr < 0)
    return ld_pair(reinterpret_cast<const T*>(fb + L::OFF_ROWLO) + (tr + R) * L::W + L::CW + cx2);
  const int gy = t.y0 + tr;
  if (t.yh && gy >= ny)
    return ld_pair(reinterpret_cast<const T*>(fb + L::OFF_ROWHI) + min(gy - ny, R - 1) * L::W +
                   L::CW + cx2);
  return ld_pair(reinterpret_cast<const T*>(fb) + (R + tr) * L::W + L::CW + cx2);
}

// Copy the wrapped halo columns of rows cy0 .. cy0+RY-1 from the column slots
// into the wide box (as fix_x_warp); `left`/`right` say which sides this warp
// reads.
template <class T, int TX, int TY, int R, int NF, int RY>
__device__ __forceinline__ void fix_x_rows(unsigned char* st, const TileInfo& t, int cy0, bool left,
                                           bool right) {
  using L = Layout<T, TX, TY, R, NF>;
  const int lane = threadIdx.x % 32;
  if (lane < R * RY) {
    const int d = lane / RY, r = lane % RY;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T* w = reinterpret_cast<T*>(st + f * L::FIELD_B);
      const T* sl = reinterpret_cast<const T*>(st + f * L::FIELD_B + L::OFF_COLL);
      const T* sr = reinterpret_cast<const T*>(st + f * L::FIELD_B + L::OFF_COLR);
      if (left) w[(R + cy0 + r) * L::W + L::CW - 1 - d] = sl[(cy0 + r) * L::CW + L::CW - 1 - d];
      if (right) w[(R + cy0 + r) * L::W + L::CW + t.nvx + d] = sr[(cy0 + r) * L::CW + d];
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
}

// One staged 2D tile on paired consumers: a warp covers a whole row group of
// TX = 64 columns, so it owns both wrapped halo column blocks of its rows.
// YW: the tile's periodic y halo wraps; all such tiles take the general
// column_pair path (2D edge tiles are a few percent of the tiles).
template <bool YW, bool WRAP, class Op, class T, int TX, int TY, int RY>
__device__ __forceinline__ void tile2d_pair(const Op& op, unsigned char* st, T* const* out, int nx,
                                            int ny, const TileInfo& t, int cx2, int cy0,
                                            double& red) {
  constexpr int R = Op::R, NF = Op::NF, NC = RY + 2 * R;
  using L = Layout<T, TX, TY, R, NF>;
  static_assert(TX == 64, "a warp of pairs spans the tile");
  if (WRAP && (t.xl || t.xr)) fix_x_rows<T, TX, TY, R, NF, RY>(st, t, cy0, t.xl, t.xr);
  F2 col[NF][NC];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const T* box = reinterpret_cast<const T*>(st + f * L::FIELD_B);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      if (YW) col[f][k] = column_pair<T, TX, TY, R, NF>(st, f, t, cy0 - R + k, cx2, ny);
      else col[f][k] = ld_pair(box + (cy0 + k) * L::W + L::CW + cx2);
    }
  }
  const bool xvalid = cx2 < t.nvx;  // nvx is even: a pair is all valid or all invalid
  const int64_t base = int64_t(t.y0 + cy0) * nx + t.x0 + cx2;
  const int64_t gclamp = int64_t(t.y0) * nx + t.x0;  // a valid pair for clamped reads
  F2 rsum(0.f);  // adjoint terms of this pair of columns, summed in FP32 per lane
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    PairAcc<T, TX, TY, R, NF, NC> acc;
#pragma unroll
    for (int f = 0; f < NF; ++f)
      acc.b[f] = reinterpret_cast<const T*>(st + f * L::FIELD_B) + (R + cy0 + r) * L::W + L::CW + cx2;
    acc.col = col;
    acc.r = r;
    acc.g = (xvalid && cy0 + r < t.nvy) ? base + int64_t(r) * nx : gclamp;
    F2 o[NF];
    F2 r1(0.f);
    op(acc, o, r1);
    if (xvalid && cy0 + r < t.nvy) {
#pragma unroll
      for (int f = 0; f < NF; ++f) st_pair(out[f] + base + int64_t(r) * nx, o[f]);
      if (Op::REDUCES) rsum = add(rsum, r1);
    }
  }
  if (Op::REDUCES) red += double(rsum.lo()) + double(rsum.hi());
}

// Box stencils on a tile whose halo wraps: each consumer warp (which spans
// the whole tile width, RY rows from cy0) rewrites the halo-ring cells of the
// wide box that its own rows read (tile rows cy0-R .. min(cy0+RY, nvy)+R-1,
// columns -R .. nvx+R-1, outside the tile's valid cells) whose global
// position lies outside the grid on periodic axes only: those take the value
// at the wrapped position.  Every other ring cell already holds the right
// value from the TMA box (in-range data, or the zero fill past a Dirichlet
// side; past an external y side the box holds the caller's rows, and only a
// corner that also crosses a periodic x side is rewritten, from the wrapped
// column of those rows).  The cells are enumerated as the 2R halo columns of
// the warp's body rows, then its halo rows over the full box width; each lane takes K cells
// per pass and issues all their loads before any store, so a warp has up to
// K * NF loads in flight.  Adjacent warps may write the same cell with the
// same value.  The proxy fence orders these shared-memory writes before the
// stage's next TMA refill; no block-wide barrier is needed.
template <class T, int TX, int TY, int R, int NF, int RY>
__device__ __forceinline__ void fill_ring_warp(unsigned char* st, const TileInfo& t,
                                               const T* const* in, int nx, int ny, int per_x,
                                               int per_y, int cy0, int ext_y = 0) {
  using L = Layout<T, TX, TY, R, NF>;
  constexpr int K = 4;
  const int lane = threadIdx.x % 32;
  if (cy0 < t.nvy) {
    const int r0 = cy0 - R, r1 = min(cy0 + RY, t.nvy) + R;  // rows [r0, r1)
    const int b0 = max(r0, 0), b1 = min(r1, t.nvy);          // body rows among them
    const int na = (b1 - b0) * 2 * R;                        // halo-column cells of the body rows
    const int nlo = max(0, -r0), nhi = max(0, r1 - t.nvy);   // halo rows above / below
    const int wr = t.nvx + 2 * R;
    const int n = na + (nlo + nhi) * wr;
    for (int c0 = 0; c0 < n; c0 += 32 * K) {
      int si[K];
      int64_t gi[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int c = c0 + k * 32 + lane;
        int tr, tc;
        if (c < na) {
          const int j = c % (2 * R);
          tr = b0 + c / (2 * R);
          tc = j < R ? j - R : t.nvx + j - R;
        } else {
          const int d = c - na, hr = d / wr;
          tr = hr < nlo ? r0 + hr : t.nvy + hr - nlo;
          tc = d % wr - R;
        }
        const int gy = t.y0 + tr, gx = t.x0 + tc;
        const bool oy = gy < 0 || gy >= ny, ox = gx < 0 || gx >= nx;
        const bool ey = (gy < 0 && (ext_y & 1)) || (gy >= ny && (ext_y & 2));
        const bool need =
            c < n && (oy || ox) && (!oy || per_y || (ey && ox)) && (!ox || per_x);
        si[k] = need ? (R + tr) * L::W + L::CW + tc : -1;
        gi[k] = need ? int64_t(oy && !ey ? wrap(gy, ny) : gy) * nx + (ox ? wrap(gx, nx) : gx) : 0;
      }
      T v[K][NF];
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int f = 0; f < NF; ++f)
          if (si[k] >= 0) v[k][f] = in[f][gi[k]];
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int f = 0; f < NF; ++f)
          if (si[k] >= 0) reinterpret_cast<T*>(st + f * L::FIELD_B)[si[k]] = v[k][f];
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
}

// Box stencils on a tile whose halo wraps on one axis only: each consumer
// warp copies the halo-ring cells its own rows read (tile rows cy0-R ..
// min(cy0+RY, nvy)+R-1) that lie past a periodic side from the slots the
// producer staged beside the box: the wrapped halo columns of the tile's rows
// and halo rows (colL / colR), or the wrapped halo rows (rowLo / rowHi).
// Every cell of a slot already holds what the boundary rule gives there
// (in-range data, the zero fill past a Dirichlet side, the caller's rows past
// an external y side), so the copy needs no further test and no global load.
template <class T, int TX, int TY, int R, int NF, int RY>
__device__ __forceinline__ void fill_ring_slots(unsigned char* st, const TileInfo& t, int ny,
                                                int cy0) {
  using L = Layout<T, TX, TY, R, NF>;
  const int lane = threadIdx.x % 32;
  if (cy0 < t.nvy) {
    const int r0 = cy0 - R, r1 = min(cy0 + RY, t.nvy) + R;  // rows [r0, r1)
    if (t.xl || t.xr) {
      // R cells on each side of every row; colL holds global columns
      // nx-CW .. nx-1, colR columns 0 .. CW-1, both for tile rows -R .. TY+R-1
      const int n = (r1 - r0) * 2 * R;
      for (int c = lane; c < n; c += 32) {
        const int tr = r0 + c / (2 * R), j = c % (2 * R);
        const bool left = j < R;
        if (left ? !t.xl : !t.xr) continue;
        const int tc = left ? j - R : t.nvx + j - R;
        const int sc = left ? L::CW + tc : tc - t.nvx;
        const int bo = (R + tr) * L::W + L::CW + tc, so = (R + tr) * L::CW + sc;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          unsigned char* fb = st + f * L::FIELD_B;
          reinterpret_cast<T*>(fb)[bo] =
              reinterpret_cast<const T*>(fb + (left ? L::OFF_COLL : L::OFF_COLR))[so];
        }
      }
    } else {
      // the halo rows among [r0, r1) past a periodic y side, columns -R .. nvx+R-1;
      // rowLo holds global rows ny-R .. ny-1, rowHi rows 0 .. R-1
      const int wr = t.nvx + 2 * R;
      for (int tr = r0; tr < r1; ++tr) {
        const int gy = t.y0 + tr;
        if (gy >= 0 && gy < ny) continue;
        const int off = gy < 0 ? L::OFF_ROWLO : L::OFF_ROWHI;
        const int sr = gy < 0 ? gy + R : gy - ny;
        for (int c = lane; c < wr; c += 32) {
          const int tc = c - R;
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            unsigned char* fb = st + f * L::FIELD_B;
            reinterpret_cast<T*>(fb)[(R + tr) * L::W + L::CW + tc] =
                reinterpret_cast<const T*>(fb + off)[sr * L::W + L::CW + tc];
          }
        }
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
}

// ------------------------------------------------------------------ 2D tiles
template <class Op, class T, int TX, int TY, int RY, int S, bool WRAP, bool PAIR>
__global__ void __launch_bounds__((PAIR ? TX / 2 : TX) * (TY / RY) + 32)
    tma2d_kernel(const __grid_constant__ TmaMaps<Op::NF> maps, const TmaParams<Op, T> p) {
  constexpr int R = Op::R, NF = Op::NF;
  using L = Layout<T, TX, TY, R, NF>;
  constexpr int NCONS = (PAIR ? TX / 2 : TX) * (TY / RY);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = align128(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * L::STAGE_B);
  uint64_t* empty = full + S;
  __shared__ volatile int abort_flag;
  __shared__ double red_scratch[NCONS / 32];

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCONS / 32);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (tid >= NCONS) {  // producer warp
    if (tid == NCONS) {
#pragma unroll
      for (int f = 0; f < NF; ++f) tma_prefetch_desc(&maps.wide[f]);
      int i = 0;
      for (int u = blockIdx.x; u < p.nunits; u += gridDim.x, ++i) {
        const int s = i % S;
        const uint32_t ph = (i / S) & 1;
        if (i >= S && !mbar_wait_bounded(&empty[s], ph ^ 1, p.err)) {
          abort_flag = 1;
          break;
        }
        if (abort_flag) break;
        const TileInfo t = classify<T, TX, TY, R>((u % p.tiles_x) * TX, (u / p.tiles_x) * TY, p.nx,
                                              p.ny, WRAP && p.per_x, WRAP && p.per_y);
        constexpr int MODE = Op::STAR ? kStageStar : kStageBox;
        issue_plane<T, TX, TY, R, NF, 2, MODE>(maps, smem + s * L::STAGE_B, &full[s], t, 0, p.nx,
                                               p.ny, p.soff);
      }
      if (abort_flag) {  // let copies already issued land before the block exits
        for (int k = max(0, i - S); k < i; ++k) mbar_wait_bounded(&full[k % S], (k / S) & 1, nullptr);
      }
    }
    return;
  }

  constexpr int CPR = PAIR ? TX / 2 : TX;  // consumer threads per row group
  const int cx = (tid % CPR) * (PAIR ? 2 : 1), cy0 = (tid / CPR) * RY, lane = tid % 32;
  double red = 0.0;
  int i = 0;
  for (int u = blockIdx.x; u < p.nunits; u += gridDim.x, ++i) {
    const int s = i % S;
    if (!mbar_wait_bounded(&full[s], (i / S) & 1, p.err) || abort_flag) {
      abort_flag = 1;
      break;
    }
    const TileInfo t = classify<T, TX, TY, R>((u % p.tiles_x) * TX, (u / p.tiles_x) * TY, p.nx,
                                              p.ny, WRAP && p.per_x, WRAP && p.per_y);
    unsigned char* st = smem + s * L::STAGE_B;
    if constexpr (!Op::STAR) {
      // Box stencil: complete the halo ring of wrapped tiles in the box, then
      // every tap (corners included) reads the box.
      static_assert(CPR == 32, "a warp spans the tile width");
      if (WRAP && (t.xl || t.xr || t.yl || t.yh)) {
        if (box_corner(t))
          fill_ring_warp<T, TX, TY, R, NF, RY>(st, t, p.in, p.nx, p.ny, p.per_x, p.per_y, cy0,
                                               p.sext);
        else
          fill_ring_slots<T, TX, TY, R, NF, RY>(st, t, p.ny, cy0);
      }
      if constexpr (PAIR)
        tile2d_pair<false, false, Op, T, TX, TY, RY>(p.op, st, p.out, p.nx, p.ny, t, cx, cy0, red);
      else
        tile2d<false, true, false, Op, T, TX, TY, RY>(p.op, st, p.out, p.nx, p.ny, t, cx, cy0, red);
    } else if constexpr (PAIR) {
      // 2D edge tiles are a few percent of the tiles: one general instance for
      // all of them keeps the persistent loop's code small.
      if (!WRAP || !(t.yl || t.yh))
        tile2d_pair<false, WRAP, Op, T, TX, TY, RY>(p.op, st, p.out, p.nx, p.ny, t, cx, cy0, red);
      else
        tile2d_pair<true, WRAP, Op, T, TX, TY, RY>(p.op, st, p.out, p.nx, p.ny, t, cx, cy0, red);
    } else {
      if (!WRAP || !(t.yl || t.yh))
        tile2d<false, true, WRAP, Op, T, TX, TY, RY>(p.op, st, p.out, p.nx, p.ny, t, cx, cy0, red);
      else
        tile2d<true, false, WRAP, Op, T, TX, TY, RY>(p.op, st, p.out, p.nx, p.ny, t, cx, cy0, red);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  if (Op::REDUCES) block_accumulate<NCONS>(red, p.partials, red_scratch);
}

// ------------------------------------------------------------------ 3D z-march
// Consumer side of the z-march for one tile.  YW: the tile's periodic y halo
// wraps, so those rows come from the row slots.  XF: x-edge tiles patch their
// wrapped halo columns per warp.
template <bool YW, bool XF, bool SIMPLE, class Op, class T, int TX, int TY, int RY, int S>
__device__ __forceinline__ void march3d(const TmaParams<Op, T>& p, unsigned char* smem,
                                        uint64_t* full, uint64_t* empty, volatile int* abort_flag,
                                        const TileInfo& t, int z0, int z1, int np, double& red) {
  using C = C_t<T>;
  constexpr int R = Op::R, NF = Op::NF, NQ = 2 * R + 1, NC = RY + 2 * R;
  using L = Layout<T, TX, TY, R, NF>;
  const int tid = threadIdx.x;
  const int cx = tid % TX, cy0 = (tid / TX) * RY, lane = tid % 32;
  const int64_t plane = int64_t(p.nx) * p.ny;
  constexpr bool simple = !YW || SIMPLE;  // strip rows never wrap
  C q[RY][NF][NQ];
  bool ok = true;

  auto release = [&](int j) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[j % S]);
  };
  // Wait for staged plane j and push its centre values onto each queue.
  auto shift_in = [&](int j) -> bool {
    const int s = j % S;
    if (!mbar_wait_bounded(&full[s], (j / S) & 1, p.err) || *abort_flag) {
      *abort_flag = 1;
      return false;
    }
    unsigned char* st = smem + s * L::STAGE_B;
    if (XF) fix_x_warp<T, TX, TY, R, NF, RY>(st, t, cx, cy0);
#pragma unroll
    for (int r = 0; r < RY; ++r)
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int k = 0; k < NQ - 1; ++k) q[r][f][k] = q[r][f][k + 1];
    if (simple) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const T* box = reinterpret_cast<const T*>(st + f * L::FIELD_B);
#pragma unroll
        for (int r = 0; r < RY; ++r) q[r][f][NQ - 1] = to_c(box[(R + cy0 + r) * L::W + L::CW + cx]);
      }
    } else {  // ragged periodic tile: strip rows past the grid edge wrap
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int r = 0; r < RY; ++r)
          q[r][f][NQ - 1] = column_value<T, TX, TY, R, NF>(st, f, t, cy0 + r, cx, p.ny, true);
    }
    return true;
  };

  for (int j = 0; j < 2 * R && ok; ++j) {
    ok = shift_in(j);
    if (ok && (j < R || j >= np - R)) release(j);  // outside [z0, z1): centres only
  }
  for (int m = 0; ok && m < z1 - z0; ++m) {
    const int jn = m + 2 * R;
    ok = shift_in(jn);
    if (!ok) break;
    const int jc = m + R;  // plane of the outputs
    const unsigned char* st = smem + (jc % S) * L::STAGE_B;
    // column registers of the output plane: strip rows from the queue, the
    // R rows on either side from the stage
    C col[NF][NC];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      edge_rows<T, TX, TY, R, NF, RY, YW>(st, f, t, cx, cy0, p.ny, simple, &col[f][0],
                                          &col[f][R + RY]);
#pragma unroll
      for (int r = 0; r < RY; ++r) col[f][R + r] = q[r][f][R];
    }
    column_rows<Op, T, TX, TY, RY, NQ, NC>(p.op, st, p.out, int64_t(z0 + m) * plane, p.nx, t, cx,
                                           cy0, col, q, red);
    release(jc);
    if (jn >= np - R) release(jn);  // above z1-1: centres only
  }
}

// Paired consumer side of the z-march (FP32/BF16 storage): each thread owns
// two adjacent columns and RY rows; the z queue and the column registers
// hold packed pairs.  A warp spans the tile width (TX = 64), so it patches
// both wrapped halo column blocks of its own rows.  ANYX: rows of any pitch
// (an odd width leaves a last column without its pair, and a pair's address
// may not be 8-byte aligned): such pairs are stored element by element.
template <bool YW, bool XF, bool SIMPLE, class Op, class T, int TX, int TY, int RY, int S,
          bool ANYX = false>
__device__ __forceinline__ void march3d_pair(const TmaParams<Op, T>& p, unsigned char* smem,
                                             uint64_t* full, uint64_t* empty,
                                             volatile int* abort_flag, const TileInfo& t, int z0,
                                             int z1, int np, double& red) {
  constexpr int R = Op::R, NF = Op::NF, NQ = 2 * R + 1, NC = RY + 2 * R;
  using L = Layout<T, TX, TY, R, NF>;
  static_assert(TX == 64, "a warp of pairs spans the tile");
  const int tid = threadIdx.x;
  const int cx2 = (tid % 32) * 2, cy0 = (tid / 32) * RY, lane = tid % 32;
  const int64_t plane = int64_t(p.nx) * p.ny;
  constexpr bool simple = !YW || SIMPLE;  // strip rows never wrap
  F2 q[RY][NF][NQ];
  bool ok = true;

  auto release = [&](int j) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[j % S]);
  };
  auto shift_in = [&](int j) -> bool {
    const int s = j % S;
    if (!mbar_wait_bounded(&full[s], (j / S) & 1, p.err) || *abort_flag) {
      *abort_flag = 1;
      return false;
    }
    unsigned char* st = smem + s * L::STAGE_B;
    if (XF) fix_x_rows<T, TX, TY, R, NF, RY>(st, t, cy0, t.xl, t.xr);
#pragma unroll
    for (int r = 0; r < RY; ++r)
#pragma unroll
      for (int f = 0; f < NF; ++f) {
#pragma unroll
        for (int k = 0; k < NQ - 1; ++k) q[r][f][k] = q[r][f][k + 1];
        if (simple)
          q[r][f][NQ - 1] = ld_pair(reinterpret_cast<const T*>(st + f * L::FIELD_B) +
                                    (R + cy0 + r) * L::W + L::CW + cx2);
        else
          q[r][f][NQ - 1] = column_pair<T, TX, TY, R, NF>(st, f, t, cy0 + r, cx2, p.ny);
      }
    return true;
  };

  for (int j = 0; j < 2 * R && ok; ++j) {
    ok = shift_in(j);
    if (ok && (j < R || j >= np - R)) release(j);  // outside [z0, z1): centres only
  }
  const bool xvalid = cx2 < t.nvx;
  for (int m = 0; ok && m < z1 - z0; ++m) {
    const int jn = m + 2 * R;
    ok = shift_in(jn);
    if (!ok) break;
    const int jc = m + R;  // plane of the outputs
    const unsigned char* st = smem + (jc % S) * L::STAGE_B;
    F2 col[NF][NC];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const T* box = reinterpret_cast<const T*>(st + f * L::FIELD_B);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        if (YW) {
          col[f][k] = column_pair<T, TX, TY, R, NF>(st, f, t, cy0 - R + k, cx2, p.ny);
          col[f][R + RY + k] = column_pair<T, TX, TY, R, NF>(st, f, t, cy0 + RY + k, cx2, p.ny);
        } else {
          col[f][k] = ld_pair(box + (cy0 + k) * L::W + L::CW + cx2);
          col[f][R + RY + k] = ld_pair(box + (cy0 + R + RY + k) * L::W + L::CW + cx2);
        }
      }
#pragma unroll
      for (int r = 0; r < RY; ++r) col[f][R + r] = q[r][f][R];
    }
    const int64_t base = int64_t(z0 + m) * plane + int64_t(t.y0 + cy0) * p.nx + t.x0 + cx2;
    const int64_t gclamp = int64_t(z0 + m) * plane + int64_t(t.y0) * p.nx + t.x0;
    F2 rsum(0.f);  // adjoint terms of this plane, summed in FP32 per lane
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      PairAcc3<T, TX, TY, R, NF, NC, NQ> acc;
#pragma unroll
      for (int f = 0; f < NF; ++f)
        acc.b[f] = reinterpret_cast<const T*>(st + f * L::FIELD_B) + (R + cy0 + r) * L::W + L::CW + cx2;
      acc.col = col;
      acc.r = r;
      acc.g = (xvalid && cy0 + r < t.nvy) ? base + int64_t(r) * p.nx : gclamp;
      acc.q = q[r];
      F2 o[NF];
      F2 r1(0.f);
      p.op(acc, o, r1);
      if (xvalid && cy0 + r < t.nvy) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          T* d = p.out[f] + base + int64_t(r) * p.nx;
          if constexpr (ANYX) {
            static_assert(sizeof(T) == 4, "element stores of FP32 pairs");
            if (cx2 + 1 < t.nvx && (reinterpret_cast<uintptr_t>(d) & 7) == 0) {
              st_pair(d, o[f]);
            } else {
              d[0] = o[f].lo();
              if (cx2 + 1 < t.nvx) d[1] = o[f].hi();
            }
          } else {
            st_pair(d, o[f]);
          }
        }
        if (Op::REDUCES) rsum = add(rsum, r1);
      }
    }
    if (Op::REDUCES) red += double(rsum.lo()) + double(rsum.hi());
    release(jc);
    if (jn >= np - R) release(jn);  // above z1-1: centres only
  }
}

// WRAP: compile the periodic-halo handling (x or y axis periodic).  Grids
// without a periodic x/y axis use the instance without it, whose consumer
// code fits the register budget of two blocks per SM.
template <class Op, class T, int TX, int TY, int RY, int S, bool WRAP, bool PAIR>
__global__ void __launch_bounds__((PAIR ? TX / 2 : TX) * (TY / RY) + 32, 2)
    tma3d_kernel(const __grid_constant__ TmaMaps<Op::NF> maps, const TmaParams<Op, T> p) {
  constexpr int R = Op::R, NF = Op::NF;
  using L = Layout<T, TX, TY, R, NF>;
  constexpr int NCONS = (PAIR ? TX / 2 : TX) * (TY / RY);
  static_assert(S >= R + 2, "ring too short for the z window");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = align128(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * L::STAGE_B);
  uint64_t* empty = full + S;
  __shared__ volatile int abort_flag;
  __shared__ double red_scratch[NCONS / 32];

  const int tid = threadIdx.x;
  const int ntiles = p.tiles_x * p.tiles_y;
  const int tile = blockIdx.x % ntiles, zc = blockIdx.x / ntiles;
  const TileInfo t = classify<T, TX, TY, R>((tile % p.tiles_x) * TX, (tile / p.tiles_x) * TY, p.nx,
                                            p.ny, WRAP && p.per_x, WRAP && p.per_y);
  const int z0 = zc * p.zchunk, z1 = min(p.nz, z0 + p.zchunk);
  const int np = (z1 - z0) + 2 * R;  // planes staged by this block

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCONS / 32);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (z0 >= z1) return;

  if (tid >= NCONS) {  // producer warp
    if (tid == NCONS) {
#pragma unroll
      for (int f = 0; f < NF; ++f) tma_prefetch_desc(&maps.wide[f]);
      int j = 0;
      for (; j < np; ++j) {
        const int s = j % S;
        const uint32_t ph = (j / S) & 1;
        if (j >= S && !mbar_wait_bounded(&empty[s], ph ^ 1, p.err)) {
          abort_flag = 1;
          break;
        }
        if (abort_flag) break;
        int z = z0 - R + j;
        if (p.per_z) z = wrap(z, p.nz);
        issue_plane<T, TX, TY, R, NF, 3>(maps, smem + s * L::STAGE_B, &full[s], t, z + p.soff, p.nx,
                                         p.ny);
      }
      if (abort_flag) {  // let copies already issued land before the block exits
        for (int k = max(0, j - S); k < j; ++k) mbar_wait_bounded(&full[k % S], (k / S) & 1, nullptr);
      }
    }
    return;
  }

  double red = 0.0;
#define LOPE_MARCH(YW, XF, SIMPLE)                                                               \
  do {                                                                                           \
    if constexpr (PAIR)                                                                          \
      march3d_pair<YW, XF, SIMPLE, Op, T, TX, TY, RY, S>(p, smem, full, empty, &abort_flag, t,   \
                                                         z0, z1, np, red);                       \
    else                                                                                         \
      march3d<YW, XF, SIMPLE, Op, T, TX, TY, RY, S>(p, smem, full, empty, &abort_flag, t, z0,    \
                                                    z1, np, red);                                \
  } while (0)
  if constexpr (WRAP) {
    const bool yw = t.yl || t.yh, xf = t.xl || t.xr;
    const bool simple = simple_y<TY>(t, p.ny);
    if (!yw) {
      if (xf) LOPE_MARCH(false, true, true);
      else LOPE_MARCH(false, false, true);
    } else if (simple) {
      if (xf) LOPE_MARCH(true, true, true);
      else LOPE_MARCH(true, false, true);
    } else {
      if (xf) LOPE_MARCH(true, true, false);
      else LOPE_MARCH(true, false, false);
    }
  } else {
    LOPE_MARCH(false, false, true);
  }
#undef LOPE_MARCH
  if (Op::REDUCES) block_accumulate<NCONS>(red, p.partials, red_scratch);
}

// ------------------------------------------------------------------ 3D z-march, copied planes
// The z-march for FP32 / FP64 grids whose rows TMA cannot stage (a row pitch
// that is not a multiple of 16 bytes): the stage ring, mbarriers and consumer
// warps of tma3d_kernel (its form without periodic-halo handling), with the
// wide box of every plane filled by NPW producer warps through 4- or 8-byte
// asynchronous copies (cp.async), which need no alignment beyond the
// element's.  Warp w stages box rows w, w + NPW, ...; lane l the box columns
// l, l + 32, l + 64, in 16- or 8-byte copies where a row's first cell is so
// aligned.  The boundary rule is applied per cell as it is staged, slowest axis first (z, then y, then x, as the direct kernel
// reads): a cell inside the grid is copied, a position past a periodic side
// is copied from the wrapped position, a cell past a Dirichlet side is stored
// with that side's value; cells no valid output reads (further than R beyond
// the tile's valid cells, outside the grid) are stored as 0.  The consumers
// then read a box that holds every halo value.  A stage's full barrier counts
// two arrivals per producer thread: one when the thread's copies into the
// stage have landed (cp.async.mbarrier.arrive.noinc) and one, with release
// semantics, after its direct stores.
template <class Op, class T, int TX, int TY, int RY, int S, bool PAIR, int NPW>
__global__ void __launch_bounds__((PAIR ? TX / 2 : TX) * (TY / RY) + 32 * NPW)
    ca3d_kernel(const __grid_constant__ Geom g, const TmaParams<Op, T> p) {
  static_assert(Op::STAR && !Op::REDUCES, "plain sweeps of star functions");
  constexpr int R = Op::R, NF = Op::NF;
  using L = Layout<T, TX, TY, R, NF>;
  constexpr int NCONS = (PAIR ? TX / 2 : TX) * (TY / RY), NP = 32 * NPW;
  constexpr int BH = TY + 2 * R, W = L::W, CW = L::CW, NK = (W + 31) / 32;
  static_assert(S >= R + 2, "ring too short for the z window");
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element copies of 4 or 8 bytes");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = align128(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * L::STAGE_B);
  uint64_t* empty = full + S;
  __shared__ volatile int abort_flag;
  __shared__ double red_scratch[NCONS / 32];

  const int tid = threadIdx.x;
  const int ntiles = p.tiles_x * p.tiles_y;
  const int tile = blockIdx.x % ntiles, zc = blockIdx.x / ntiles;
  const TileInfo t = classify<T, TX, TY, R>((tile % p.tiles_x) * TX, (tile / p.tiles_x) * TY, p.nx,
                                            p.ny, 0, 0);
  const int z0 = zc * p.zchunk, z1 = min(p.nz, z0 + p.zchunk);
  const int np = (z1 - z0) + 2 * R;  // planes staged by this block

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 2 * NP);
      mbar_init(&empty[s], NCONS / 32);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (z0 >= z1) return;

  if (tid >= NCONS) {  // producer warps
    constexpr int NRW = (BH + NPW - 1) / NPW;  // box rows per producer warp
    const int pw = (tid - NCONS) / 32, lane = tid % 32;
    const int64_t plane = int64_t(p.nx) * p.ny;
    // This lane's columns (the same on every row and plane): 0 copy from
    // gcol, 1 / 2 the low / high x side's Dirichlet value, -1 unused (0).
    int gcol[NK], ccode[NK];
    // every box column inside the grid: rows are copied as runs of consecutive cells
    const bool all_copy = t.x0 - CW >= 0 && t.x0 - CW + W <= p.nx;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      const int tc = lane + 32 * k - CW, gx = t.x0 + tc;
      gcol[k] = 0;
      if (lane + 32 * k >= W) {
        ccode[k] = -1;
        continue;
      }
      if (gx >= 0 && gx < p.nx) {
        ccode[k] = 0;
        gcol[k] = gx;
      } else if (tc >= -R && tc < t.nvx + R) {
        const int xx = axis_index(gx, p.nx, g.bc[2][0], g.bc[2][1]);
        ccode[k] = xx < 0 ? -xx : 0;
        gcol[k] = xx < 0 ? 0 : xx;
      } else {
        ccode[k] = -1;
      }
    }
    // This warp's rows (the same on every plane): the element offset of the
    // source row in its plane, or -1 / -2 past the low / high y Dirichlet
    // side, or -3 for a row no output reads.
    int64_t yrow[NRW];
#pragma unroll
    for (int i = 0; i < NRW; ++i) {
      const int br = pw + NPW * i, tr = br - R, gy = t.y0 + tr;
      int yy = -3;
      if (br < BH) {
        if (gy >= 0 && gy < p.ny) yy = gy;
        else if (tr >= -R && tr < t.nvy + R) yy = axis_index(gy, p.ny, g.bc[1][0], g.bc[1][1]);
      }
      yrow[i] = yy >= 0 ? int64_t(yy) * p.nx : int64_t(yy);
    }
    const T vx0 = T(g.bval[2][0]), vx1 = T(g.bval[2][1]);
    const T vy0 = T(g.bval[1][0]), vy1 = T(g.bval[1][1]);
    // a row of one value: every cell the outputs read, 0 elsewhere
    auto fill_row = [&](T* brow, T v) {
#pragma unroll
      for (int k = 0; k < NK; ++k)
        if (lane + 32 * k < W) brow[lane + 32 * k] = ccode[k] < 0 ? T(0) : v;
    };
    for (int j = 0; j < np; ++j) {
      const int s = j % S;
      if (j >= S && !mbar_wait_bounded(&empty[s], ((j / S) & 1) ^ 1, p.err)) {
        abort_flag = 1;
        break;
      }
      if (abort_flag) break;
      const int zz = axis_index(z0 - R + j, p.nz, g.bc[0][0], g.bc[0][1]);
      unsigned char* st = smem + s * L::STAGE_B;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        T* box = reinterpret_cast<T*>(st + f * L::FIELD_B);
        const uint32_t sbox = smem_u32(box);
        if (zz < 0) {  // a plane past a Dirichlet z side: its value (z decides first)
          const T v = T(g.bval[0][-zz - 1]);
#pragma unroll
          for (int i = 0; i < NRW; ++i)
            if (pw + NPW * i < BH) fill_row(box + (pw + NPW * i) * W, v);
          continue;
        }
        const T* src = p.in[f] + int64_t(zz) * plane;
#pragma unroll
        for (int i = 0; i < NRW; ++i) {
          const int br = pw + NPW * i;
          if (br >= BH) break;
          T* brow = box + br * W;
          const int64_t yo = yrow[i];
          if (yo < 0) {  // a y Dirichlet side decides before x
            fill_row(brow, yo == -3 ? T(0) : yo == -1 ? vy0 : vy1);
            continue;
          }
          const T* row = src + yo;
          const uint32_t d = sbox + uint32_t(br * W + lane) * uint32_t(sizeof(T));
          if (all_copy) {
            // the row's cells are consecutive in memory: 16- or 8-byte copies
            // where the row's first cell is so aligned (the box row is)
            const T* r0 = row + (t.x0 - CW);
            const uint32_t drow = sbox + uint32_t(br * W) * uint32_t(sizeof(T));
            const unsigned mis = unsigned(reinterpret_cast<uintptr_t>(r0)) & 15u;
            if (mis == 0) {
              constexpr int E = 16 / int(sizeof(T)), NV = W / E;
              static_assert(W % E == 0 && NV <= 32, "a box row in 16-byte copies");
              if (lane < NV) cp_async_16(drow + 16u * lane, r0 + E * lane);
            } else if (sizeof(T) == 4 && (mis & 7u) == 0) {
              constexpr int NV = W / 2;
#pragma unroll
              for (int k = 0; k * 32 < NV; ++k)
                if (lane + 32 * k < NV) cp_async_elem<8>(drow + 8u * (lane + 32 * k), r0 + 2 * (lane + 32 * k));
            } else {
#pragma unroll
              for (int k = 0; k < NK; ++k)
                if (lane + 32 * k < W) cp_async_elem<int(sizeof(T))>(d + 32u * k * sizeof(T), r0 + lane + 32 * k);
            }
          } else {
#pragma unroll
            for (int k = 0; k < NK; ++k) {
              if (lane + 32 * k >= W) continue;
              if (ccode[k] == 0) cp_async_elem<int(sizeof(T))>(d + 32u * k * sizeof(T), row + gcol[k]);
              else brow[lane + 32 * k] = ccode[k] < 0 ? T(0) : ccode[k] == 1 ? vx0 : vx1;
            }
          }
        }
      }
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[s]))
                   : "memory");
      mbar_arrive(&full[s]);
    }
    cp_async_wait_all();  // this thread's copies land before it leaves
    return;
  }

  double red = 0.0;
  if constexpr (PAIR)
    march3d_pair<false, false, true, Op, T, TX, TY, RY, S, true>(p, smem, full, empty, &abort_flag,
                                                                 t, z0, z1, np, red);
  else
    march3d<false, false, true, Op, T, TX, TY, RY, S>(p, smem, full, empty, &abort_flag, t, z0, z1,
                                                      np, red);
  if (Op::REDUCES) block_accumulate<NCONS>(red, p.partials, red_scratch);
}

// ------------------------------------------------------------------ 3D z-march, two sweeps
// Temporal blocking of depth 2 on the paired z-march: one launch applies the
// local function twice (the fusion latitude of Sec. 3.5) while staging each
// input plane from HBM once, so a sweep costs half the HBM bytes of the
// one-sweep march.  For radius-1 star functions of one field on grids whose x
// and y sides are Dirichlet 0: the TMA zero fill is then the halo of the
// input, and the intermediate state u1 is set to the halo value 0 outside the
// grid (a periodic z axis is staged from wrapped planes).
//
// Each input plane is staged with a 2-row / 16-byte-column halo.  Every
// consumer warp owns RY rows x 64 columns of the tile (pairs of columns per
// lane) and keeps, in a private three-plane ring of shared-memory slots, u1
// on its rows, the row above and the row below them (computed again by the
// neighbouring warps: no block-wide barrier) and the column pairs just left
// and right of the tile.  Per staged plane j a warp
//   * pushes u0(j) of its cells onto its register queue,
//   * computes u1 at plane j-1: own cells from the queue and the staged box,
//     the extra rows and columns from three staged planes, rounded to the
//     storage precision as a stored sweep would be (bitwise the one-sweep
//     result), and writes them to its slot,
//   * computes u2 at plane j-2 from the u1 register queue and the slot of
//     plane j-2, and stores it.
template <bool B> struct BoolTag { static constexpr bool value = B; };

template <class S_, int WS>
struct Tb2Acc {  // x taps from a buffer of row stride WS, y taps and centre from column registers
  const S_* b;
  const F2* col;  // col[1 + dy]
  F2 zm, zp;      // the planes below and above
  __device__ __forceinline__ F2 operator()(int, int dx, int dy, int dz) const {
    if (dz != 0) return dz < 0 ? zm : zp;
    if (dx == 0) return col[1 + dy];
    const F2 c = col[1];
    if (dx == -1) return F2::make(ld_pair(b - 2).hi(), c.lo());
    return F2::make(c.hi(), ld_pair(b + 2).lo());
  }
  __device__ __forceinline__ int64_t gidx() const { return 0; }
};

template <int V> struct IntTag { static constexpr int value = V; };

template <class S_, int WS>
struct Tb2SmemAcc {  // every tap from three staged planes (centre c, below lo, above hi)
  const S_* c;
  const S_* lo;
  const S_* hi;
  __device__ __forceinline__ F2 operator()(int, int dx, int dy, int dz) const {
    if (dz == -1) return ld_pair(lo);
    if (dz == 1) return ld_pair(hi);
    const S_* rb = c + dy * WS;
    if (dx == 0) return ld_pair(rb);
    if (dx == -1) return F2::make(ld_pair(rb - 2).hi(), ld_pair(rb).lo());
    return F2::make(ld_pair(rb).hi(), ld_pair(rb + 2).lo());
  }
  __device__ __forceinline__ int64_t gidx() const { return 0; }
};

__device__ __forceinline__ void st_pair_f(float* p, F2 v) { *reinterpret_cast<uint64_t*>(p) = v.v; }

// The value a stored sweep would hold (identity for FP32; BF16 rounds).
template <class T> __device__ __forceinline__ F2 stored_pair(F2 v) { return v; }
template <> __device__ __forceinline__ F2 stored_pair<__nv_bfloat16>(F2 v) {
  return F2::make(__bfloat162float(__float2bfloat16_rn(v.lo())),
                  __bfloat162float(__float2bfloat16_rn(v.hi())));
}

template <int TX, int TY, int RY> struct Tb2Slots {
  static constexpr int W1 = TX + 8;     // columns -4 .. TX+3 (floats)
  static constexpr int SR = RY + 2;     // tile rows cy0-1 .. cy0+RY
  static constexpr int SLOT = SR * W1;  // floats per plane slot
  static constexpr int NW = TY / RY;    // consumer warps
  static constexpr uint32_t BYTES = uint32_t(NW) * 3 * SLOT * sizeof(float);
};

template <class Op, class T, int TX, int TY, int RY, int S>
__global__ void __launch_bounds__((TX / 2) * (TY / RY) + 32, 1)
    tma3d_tb2_kernel(const __grid_constant__ TmaMaps<1> maps, const TmaParams<Op, T> p) {
  static_assert(Op::R == 1 && Op::NF == 1 && Op::STAR && TX == 64, "radius-1 star, one field");
  constexpr int H = 2;  // staged halo rows: two sweeps of radius 1
  using L = Layout<T, TX, TY, H, 1>;
  using SL = Tb2Slots<TX, TY, RY>;
  constexpr int NCONS = 32 * SL::NW, W = L::W, CW = L::CW, W1 = SL::W1;
  constexpr uint32_t STAGE = L::OFF_COLL;  // the wide box alone (no wrapped-halo slots)
  static_assert(S >= 4, "ring too short for three planes and one in flight");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = align128(smem_raw);
  float* slots = reinterpret_cast<float*>(smem + S * STAGE);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * STAGE + SL::BYTES);
  uint64_t* empty = full + S;
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x;
  const int ntiles = p.tiles_x * p.tiles_y;
  const int tile = blockIdx.x % ntiles, zc = blockIdx.x / ntiles;
  const TileInfo t = classify<T, TX, TY, H>((tile % p.tiles_x) * TX, (tile / p.tiles_x) * TY, p.nx,
                                            p.ny, 0, 0);
  const int z0 = zc * p.zchunk, z1 = min(p.nz, z0 + p.zchunk);
  const int np = (z1 - z0) + 2 * H;  // planes staged by this block

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCONS / 32);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (z0 >= z1) return;

  if (tid >= NCONS) {  // producer warp
    if (tid == NCONS) {
      tma_prefetch_desc(&maps.wide[0]);
      int j = 0;
      for (; j < np; ++j) {
        const int s = j % S;
        if (j >= S && !mbar_wait_bounded(&empty[s], ((j / S) & 1) ^ 1, p.err)) {
          abort_flag = 1;
          break;
        }
        if (abort_flag) break;
        int z = z0 - H + j;
        if (p.per_z) z = wrap(z, p.nz);
        issue_plane<T, TX, TY, H, 1, 3, kStageWide>(maps, smem + s * STAGE, &full[s], t, z, p.nx, p.ny);
      }
      if (abort_flag) {  // let copies already issued land before the block exits
        for (int k = max(0, j - S); k < j; ++k) mbar_wait_bounded(&full[k % S], (k / S) & 1, nullptr);
      }
    }
    return;
  }

  const int lane = tid % 32, warp = tid / 32;
  const int cx2 = lane * 2, cy0 = warp * RY;
  float* myslots = slots + warp * 3 * SL::SLOT;
  const int64_t plane = int64_t(p.nx) * p.ny;
  const bool xin = t.x0 + cx2 < p.nx;  // nx is even: a pair is all in or all out
  auto stage = [&](int j) { return reinterpret_cast<const T*>(smem + (j % S) * STAGE); };
  auto release = [&](int j) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[j % S]);
  };
  // inside the grid in x and y (tile row tr, tile column tc of a pair)
  auto inside = [&](int tr, int tc) {
    const int gy = t.y0 + tr, gx = t.x0 + tc;
    return gy >= 0 && gy < p.ny && gx >= 0 && gx < p.nx;
  };
  // A warp whose cells, extra rows or side columns leave the grid in x or y
  // masks them to the Dirichlet value 0; the others compile without masks.
  const bool edge = t.x0 == 0 || t.y0 + cy0 == 0 || t.x0 + TX + 2 > p.nx ||
                    t.y0 + cy0 + RY + 1 > p.ny;
  T* outp = p.out[0] + int64_t(z0) * plane + int64_t(t.y0 + cy0) * p.nx + t.x0 + cx2;

  // Register queues, rotated by renaming: the plane loop is unrolled by 3, so
  // plane j's u0 sits in q0[j % 3] and u1 of plane j in q1[j % 3].
  F2 q0[3][RY];
  F2 q1[3][RY];
  bool ok = true;
  auto step = [&](auto ph_tag, auto edge_tag, int j) {
    constexpr int PH = decltype(ph_tag)::value;  // j % 3
    constexpr bool EDGE = decltype(edge_tag)::value;
    constexpr int P1 = (PH + 2) % 3, P2 = (PH + 1) % 3;  // (j-1) % 3, (j-2) % 3
    if (!mbar_wait_bounded(&full[j % S], (j / S) & 1, p.err) || abort_flag) {
      abort_flag = 1;
      ok = false;
      return;
    }
    const T* bj = stage(j);
#pragma unroll
    for (int r = 0; r < RY; ++r) q0[PH][r] = ld_pair(bj + (H + cy0 + r) * W + CW + cx2);
    if (j < 2) return;
    // ---- u1 at plane j-1
    const int zg = z0 - H + (j - 1);
    const bool zout = !p.per_z && (zg < 0 || zg >= p.nz);  // Dirichlet-0 plane: u1 = 0
    const T* bc = stage(j - 1);
    const T* blo = stage(j - 2);
    float* s1 = myslots + P1 * SL::SLOT;
    if (zout) {
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        q1[P1][r] = F2(0.f);
        st_pair_f(s1 + (1 + r) * W1 + 4 + cx2, F2(0.f));
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) st_pair_f(s1 + (e ? RY + 1 : 0) * W1 + 4 + cx2, F2(0.f));
      if (lane < 2 * SL::SR)
        st_pair_f(s1 + (lane >> 1) * W1 + 4 + ((lane & 1) ? TX : -2), F2(0.f));
    } else {
      F2 col[RY + 2];
      col[0] = ld_pair(bc + (H + cy0 - 1) * W + CW + cx2);
      col[RY + 1] = ld_pair(bc + (H + cy0 + RY) * W + CW + cx2);
#pragma unroll
      for (int r = 0; r < RY; ++r) col[1 + r] = q0[P1][r];
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        Tb2Acc<T, W> acc{bc + (H + cy0 + r) * W + CW + cx2, col + r, q0[P2][r], q0[PH][r]};
        F2 o[1];
        F2 unused(0.f);
        p.op(acc, o, unused);
        F2 v = stored_pair<T>(o[0]);
        if constexpr (EDGE)
          if (!(xin && t.y0 + cy0 + r < p.ny)) v = F2(0.f);
        q1[P1][r] = v;
        st_pair_f(s1 + (1 + r) * W1 + 4 + cx2, v);
      }
      // the rows above and below the warp's rows, and the column pairs beside
      // the tile on all of them, from the three staged planes
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int tr = e ? cy0 + RY : cy0 - 1;
        const int off = (H + tr) * W + CW + cx2;
        Tb2SmemAcc<T, W> acc{bc + off, blo + off, bj + off};
        F2 o[1];
        F2 unused(0.f);
        p.op(acc, o, unused);
        F2 v = stored_pair<T>(o[0]);
        if constexpr (EDGE)
          if (!inside(tr, cx2)) v = F2(0.f);
        st_pair_f(s1 + (e ? RY + 1 : 0) * W1 + 4 + cx2, v);
      }
      if (lane < 2 * SL::SR) {
        const int row = lane >> 1, tc = (lane & 1) ? TX : -2;
        const int tr = cy0 - 1 + row;
        const int off = (H + tr) * W + CW + tc;
        Tb2SmemAcc<T, W> acc{bc + off, blo + off, bj + off};
        F2 o[1];
        F2 unused(0.f);
        p.op(acc, o, unused);
        F2 v = stored_pair<T>(o[0]);
        if constexpr (EDGE)
          if (!inside(tr, tc)) v = F2(0.f);
        st_pair_f(s1 + row * W1 + 4 + tc, v);
      }
    }
    release(j - 2);  // u0 plane j-2 is no longer read (the __syncwarp also publishes s1)
    if (j < 4) return;
    // ---- u2 at plane j-2 (output plane z0 + j - 4)
    const float* s2 = myslots + P2 * SL::SLOT;
    F2 col[RY + 2];
    col[0] = ld_pair(s2 + 4 + cx2);
    col[RY + 1] = ld_pair(s2 + (RY + 1) * W1 + 4 + cx2);
#pragma unroll
    for (int r = 0; r < RY; ++r) col[1 + r] = q1[P2][r];
    T* o_plane = outp + int64_t(j - 4) * plane;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      Tb2Acc<float, W1> acc{s2 + (1 + r) * W1 + 4 + cx2, col + r, q1[PH][r], q1[P1][r]};
      F2 o[1];
      F2 unused(0.f);
      p.op(acc, o, unused);
      if (!EDGE || (xin && t.y0 + cy0 + r < p.ny)) st_pair(o_plane + int64_t(r) * p.nx, o[0]);
    }
  };
  auto march = [&](auto edge_tag) {
    for (int j0 = 0; j0 < np && ok; j0 += 3) {
      step(IntTag<0>(), edge_tag, j0);
      if (ok && j0 + 1 < np) step(IntTag<1>(), edge_tag, j0 + 1);
      if (ok && j0 + 2 < np) step(IntTag<2>(), edge_tag, j0 + 2);
    }
  };
  if (edge) march(BoolTag<true>());
  else march(BoolTag<false>());
  if (ok) {
    release(np - 2);
    release(np - 1);
  }
}

// Named barrier `id` over `nthreads` threads that also ORs a predicate over
// them: every thread gets the same answer.
__device__ __forceinline__ bool bar_or(int id, int nthreads, bool pred) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "barrier.cta.red.or.pred q, %2, %3, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(int(pred)), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

// The same two-sweep z-march with the u1 planes shared by the block: every
// consumer warp computes u1 on its RY rows of the tile and the block shares
// the R-wide ring around the tile (the rows above and below, the column pairs
// beside), so no row is computed twice; the warps meet at named barrier 1 once
// per plane, between writing u1 of plane j-1 and reading it for u2.  Three
// plane slots rotate: slot (j-1) % 3 is written at plane j, read at plane j+1
// and written again at plane j+3, after every warp has passed the barrier of
// plane j+2.  The barrier ORs the warps' wait failures, so all leave together.
template <class Op, class T, int TX, int TY, int RY, int S>
__global__ void __launch_bounds__((TX / 2) * (TY / RY) + 32, 1)
    tma3d_tb2s_kernel(const __grid_constant__ TmaMaps<1> maps, const TmaParams<Op, T> p) {
  static_assert(Op::R == 1 && Op::NF == 1 && Op::STAR && TX == 64, "radius-1 star, one field");
  constexpr int H = 2;
  using L = Layout<T, TX, TY, H, 1>;
  constexpr int NW = TY / RY, NCONS = 32 * NW, W = L::W, CW = L::CW;
  constexpr int W1 = TX + 8, SR = TY + 2;  // slot: rows -1 .. TY, columns -4 .. TX+3
  constexpr int SLOT = SR * W1;
  constexpr uint32_t STAGE = L::OFF_COLL;
  constexpr int NRING = 2 * 32 + 2 * SR;  // rows -1 and TY; column pairs -2 and TX on rows -1..TY
  static_assert(S >= 4, "ring too short for three planes and one in flight");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = align128(smem_raw);
  float* slots = reinterpret_cast<float*>(smem + S * STAGE);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * STAGE + 3 * SLOT * 4);
  uint64_t* empty = full + S;
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x;
  const int ntiles = p.tiles_x * p.tiles_y;
  const int tile = blockIdx.x % ntiles, zc = blockIdx.x / ntiles;
  const TileInfo t = classify<T, TX, TY, H>((tile % p.tiles_x) * TX, (tile / p.tiles_x) * TY, p.nx,
                                            p.ny, 0, 0);
  const int z0 = zc * p.zchunk, z1 = min(p.nz, z0 + p.zchunk);
  const int np = (z1 - z0) + 2 * H;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCONS / 32);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (z0 >= z1) return;

  if (tid >= NCONS) {  // producer warp
    if (tid == NCONS) {
      tma_prefetch_desc(&maps.wide[0]);
      int j = 0;
      for (; j < np; ++j) {
        const int s = j % S;
        if (j >= S && !mbar_wait_bounded(&empty[s], ((j / S) & 1) ^ 1, p.err)) {
          abort_flag = 1;
          break;
        }
        if (abort_flag) break;
        int z = z0 - H + j;
        if (p.per_z) z = wrap(z, p.nz);
        issue_plane<T, TX, TY, H, 1, 3, kStageWide>(maps, smem + s * STAGE, &full[s], t, z, p.nx, p.ny);
      }
      if (abort_flag) {
        for (int k = max(0, j - S); k < j; ++k) mbar_wait_bounded(&full[k % S], (k / S) & 1, nullptr);
      }
    }
    return;
  }

  const int lane = tid % 32, warp = tid / 32;
  const int cx2 = lane * 2, cy0 = warp * RY;
  const int64_t plane = int64_t(p.nx) * p.ny;
  const bool xin = t.x0 + cx2 < p.nx;
  auto stage = [&](int j) { return reinterpret_cast<const T*>(smem + (j % S) * STAGE); };
  auto inside = [&](int tr, int tc) {
    const int gy = t.y0 + tr, gx = t.x0 + tc;
    return gy >= 0 && gy < p.ny && gx >= 0 && gx < p.nx;
  };
  const bool edge = t.x0 == 0 || t.y0 == 0 || t.x0 + TX + 2 > p.nx || t.y0 + TY + 1 > p.ny;
  T* outp = p.out[0] + int64_t(z0) * plane + int64_t(t.y0 + cy0) * p.nx + t.x0 + cx2;

  F2 q0[3][RY];
  F2 q1[3][RY];
  bool ok = true;       // changes only at a barrier: the same in every warp
  bool failed = false;  // this warp's waits so far
  auto step = [&](auto ph_tag, auto edge_tag, int j) {
    constexpr int PH = decltype(ph_tag)::value;
    constexpr bool EDGE = decltype(edge_tag)::value;
    constexpr int P1 = (PH + 2) % 3, P2 = (PH + 1) % 3;
    const bool got = !failed && mbar_wait_bounded(&full[j % S], (j / S) & 1, p.err) && !abort_flag;
    failed = !got;
    const T* bj = stage(j);
    if (got) {
#pragma unroll
      for (int r = 0; r < RY; ++r) q0[PH][r] = ld_pair(bj + (H + cy0 + r) * W + CW + cx2);
    }
    if (j < 2) return;  // a failure here is reported at the next barrier
    // ---- u1 at plane j-1
    const int zg = z0 - H + (j - 1);
    const bool zout = !p.per_z && (zg < 0 || zg >= p.nz);
    const T* bc = stage(j - 1);
    const T* blo = stage(j - 2);
    float* s1 = slots + P1 * SLOT;
    if (got) {
      if (zout) {
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          q1[P1][r] = F2(0.f);
          st_pair_f(s1 + (1 + cy0 + r) * W1 + 4 + cx2, F2(0.f));
        }
        for (int c = tid; c < NRING; c += NCONS) {
          const int tr = c < 64 ? ((c >> 5) ? TY : -1) : (c - 64) / 2 - 1;
          const int tc = c < 64 ? (c & 31) * 2 : (((c - 64) & 1) ? TX : -2);
          st_pair_f(s1 + (1 + tr) * W1 + 4 + tc, F2(0.f));
        }
      } else {
        F2 col[RY + 2];
        col[0] = ld_pair(bc + (H + cy0 - 1) * W + CW + cx2);
        col[RY + 1] = ld_pair(bc + (H + cy0 + RY) * W + CW + cx2);
#pragma unroll
        for (int r = 0; r < RY; ++r) col[1 + r] = q0[P1][r];
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          Tb2Acc<T, W> acc{bc + (H + cy0 + r) * W + CW + cx2, col + r, q0[P2][r], q0[PH][r]};
          F2 o[1];
          F2 unused(0.f);
          p.op(acc, o, unused);
          F2 v = stored_pair<T>(o[0]);
          if constexpr (EDGE)
            if (!(xin && t.y0 + cy0 + r < p.ny)) v = F2(0.f);
          q1[P1][r] = v;
          st_pair_f(s1 + (1 + cy0 + r) * W1 + 4 + cx2, v);
        }
        for (int c = tid; c < NRING; c += NCONS) {
          const int tr = c < 64 ? ((c >> 5) ? TY : -1) : (c - 64) / 2 - 1;
          const int tc = c < 64 ? (c & 31) * 2 : (((c - 64) & 1) ? TX : -2);
          const int off = (H + tr) * W + CW + tc;
          Tb2SmemAcc<T, W> acc{bc + off, blo + off, bj + off};
          F2 o[1];
          F2 unused(0.f);
          p.op(acc, o, unused);
          F2 v = stored_pair<T>(o[0]);
          if constexpr (EDGE)
            if (!inside(tr, tc)) v = F2(0.f);
          st_pair_f(s1 + (1 + tr) * W1 + 4 + tc, v);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[(j - 2) % S]);  // u0 plane j-2 is no longer read
    }
    if (bar_or(1, NCONS, !got)) {  // u1 of plane j-1 complete, or some warp gave up
      abort_flag = 1;
      ok = false;
      return;
    }
    if (j < 4) return;
    // ---- u2 at plane j-2 (output plane z0 + j - 4)
    const float* s2 = slots + P2 * SLOT;
    F2 col[RY + 2];
    col[0] = ld_pair(s2 + cy0 * W1 + 4 + cx2);
    col[RY + 1] = ld_pair(s2 + (cy0 + RY + 1) * W1 + 4 + cx2);
#pragma unroll
    for (int r = 0; r < RY; ++r) col[1 + r] = q1[P2][r];
    T* o_plane = outp + int64_t(j - 4) * plane;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      Tb2Acc<float, W1> acc{s2 + (1 + cy0 + r) * W1 + 4 + cx2, col + r, q1[PH][r], q1[P1][r]};
      F2 o[1];
      F2 unused(0.f);
      p.op(acc, o, unused);
      if (!EDGE || (xin && t.y0 + cy0 + r < p.ny)) st_pair(o_plane + int64_t(r) * p.nx, o[0]);
    }
  };
  auto march = [&](auto edge_tag) {
    for (int j0 = 0; j0 < np && ok; j0 += 3) {
      step(IntTag<0>(), edge_tag, j0);
      if (ok && j0 + 1 < np) step(IntTag<1>(), edge_tag, j0 + 1);
      if (ok && j0 + 2 < np) step(IntTag<2>(), edge_tag, j0 + 2);
    }
  };
  if (edge) march(BoolTag<true>());
  else march(BoolTag<false>());
  if (ok) {
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&empty[(np - 2) % S]);
      mbar_arrive(&empty[(np - 1) % S]);
    }
  }
}

// ------------------------------------------------------------------ 2D tiles, two sweeps
// Temporal blocking of depth 2 on the 2D TMA tiles (radius-1 and radius-2
// functions of one or more fields, star or box, paired consumers): each 64 x
// TY tile is staged once with a 2R-row / 16-byte-column halo, the first sweep
// u1 = E(u0) is computed on the tile plus an R-wide ring (the rows above and
// below it and the column pairs beside it, corners included for box
// functions: every cell the second sweep reads) into a shared-memory buffer
// per field, and the second sweep writes the tile.
// Periodic sides: on tiles whose staged halo crosses one, the consumers first
// rewrite the cells past it from the wrapped global coordinates (the TMA box
// holds zeros there), so the staged window is the periodic extension and u1 on
// the ring is the periodic value.  Dirichlet sides (value 0): the zero fill is
// the halo of u0 and u1 is set to 0 past them.  u1 is rounded to the storage
// precision, so the result is bitwise that of two one-sweep launches.
template <class S_, int WS, int FS = 0>
struct Smem2Acc {  // every tap of a star function from staged 2D buffers (field stride FS)
  const S_* c;
  __device__ __forceinline__ F2 operator()(int f, int dx, int dy, int) const {
    const S_* rb = c + f * FS + dy * WS;
    if (dx == 0) return ld_pair(rb);
    if (dx == -2) return ld_pair(rb - 2);
    if (dx == 2) return ld_pair(rb + 2);
    if (dx == -1) return F2::make(ld_pair(rb - 2).hi(), ld_pair(rb).lo());
    return F2::make(ld_pair(rb).hi(), ld_pair(rb + 2).lo());
  }
  __device__ __forceinline__ int64_t gidx() const { return 0; }
};

// Shared-memory sizes of the two-sweep 2D tiles: a stage holds the wide box of
// every field (one field: the box alone; several: at the field stride of the
// stage layout, which issue_plane writes), a u1 buffer TY + 2R rows of
// TX + 8 FP32 columns per field.
template <class T, int TY, int R, int NF>
struct Tb2Mem2D {
  using L = Layout<T, 64, TY, 2 * R, NF>;
  static constexpr uint32_t STAGE = NF == 1 ? L::OFF_COLL : NF * L::FIELD_B;
  static constexpr int W1 = 64 + 8;
  static constexpr uint32_t U1B = (uint32_t(TY + 2 * R) * W1 * 4 + 127) / 128 * 128;
};

template <class Op, class T, int TY, int RY, int S, bool WRAP>
__global__ void __launch_bounds__((TY / RY) * 32 + 32, 1)
    tma2d_tb2_kernel(const __grid_constant__ TmaMaps<Op::NF> maps, const TmaParams<Op, T> p) {
  constexpr int TX = 64, R = Op::R, H = 2 * R, NF = Op::NF;
  static_assert(R <= 2 && NF <= kMaxFields, "radius <= 2");
  using L = Layout<T, TX, TY, H, NF>;
  using M = Tb2Mem2D<T, TY, R, NF>;
  constexpr int NW = TY / RY, NCONS = 32 * NW, W = L::W, CW = L::CW, NC = RY + 2 * R;
  static_assert(CW >= H, "the staged columns cover two sweeps of the radius");
  constexpr int W1 = M::W1;              // u1 row: columns -4 .. TX+3 (floats)
  constexpr uint32_t STAGE = M::STAGE;
  constexpr uint32_t U1B = M::U1B;
  constexpr int FB = int(L::FIELD_B / sizeof(T)), FU = int(U1B / 4);  // field strides
  // ring pairs: 2R rows x 32, 2 columns x TY rows, and for box functions the
  // 2R x 2 corner pairs
  constexpr int NRING = 2 * R * 32 + 2 * TY + (Op::STAR ? 0 : 4 * R);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = align128(smem_raw);
  float* u1s = reinterpret_cast<float*>(smem + S * STAGE);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * STAGE + 2 * NF * U1B);
  uint64_t* empty = full + S;
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCONS / 32);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (tid >= NCONS) {  // producer warp
    if (tid == NCONS) {
#pragma unroll
      for (int f = 0; f < NF; ++f) tma_prefetch_desc(&maps.wide[f]);
      int i = 0;
      for (int u = blockIdx.x; u < p.nunits; u += gridDim.x, ++i) {
        const int s = i % S;
        if (i >= S && !mbar_wait_bounded(&empty[s], ((i / S) & 1) ^ 1, p.err)) {
          abort_flag = 1;
          break;
        }
        if (abort_flag) break;
        const TileInfo t = classify<T, TX, TY, H>((u % p.tiles_x) * TX, (u / p.tiles_x) * TY, p.nx,
                                                  p.ny, 0, 0);
        issue_plane<T, TX, TY, H, NF, 2, kStageWide>(maps, smem + s * STAGE, &full[s], t, 0, p.nx,
                                                     p.ny);
      }
      if (abort_flag) {  // let copies already issued land before the block exits
        for (int k = max(0, i - S); k < i; ++k) mbar_wait_bounded(&full[k % S], (k / S) & 1, nullptr);
      }
    }
    return;
  }

  const int lane = tid % 32, warp = tid / 32;
  const int cx2 = lane * 2, cy0 = warp * RY;
  const bool per_x = WRAP && p.per_x, per_y = WRAP && p.per_y;
  // The consumer warps meet at named barrier 1 (NCONS threads) after the
  // periodic rewrite and after the first sweep.  A warp whose bounded wait
  // gave up skips the work but still reaches both barriers; the second one
  // ORs the failures, so every warp leaves the loop together (no warp is
  // left waiting at a barrier).
  int i = 0;
  for (int u = blockIdx.x; u < p.nunits; u += gridDim.x, ++i) {
    const int s = i % S;
    const bool got = mbar_wait_bounded(&full[s], (i / S) & 1, p.err) && !abort_flag;
    const int x0 = (u % p.tiles_x) * TX, y0 = (u / p.tiles_x) * TY;
    T* box = reinterpret_cast<T*>(smem + s * STAGE);  // field f at box + f * FB
    float* u1 = u1s + (i & 1) * NF * FU;               // field f at u1 + f * FU
    // cells of this tile's window past a grid side; the others compute unmasked
    const bool edge = x0 < CW || x0 + TX + CW > p.nx || y0 < H || y0 + TY + H > p.ny;
    if (WRAP && edge && (per_x || per_y)) {
      // the staged window past a periodic side: the wrapped values.  Only the
      // strips past a side are visited: box columns [0, cl) and [cr, W) over
      // all rows, box rows [0, rt) and [rb, BH) over the columns between.
      constexpr int BH = TY + 2 * H;
      const int cl = max(0, min(W, CW - x0)), cr = max(cl, min(W, p.nx - (x0 - CW)));
      const int rt = max(0, min(BH, H - y0)), rb = max(rt, min(BH, p.ny - (y0 - H)));
      auto fix = [&](int br, int bcol) {
        const int gy = y0 - H + br, gx = x0 - CW + bcol;
        const bool oy = gy < 0 || gy >= p.ny, ox = gx < 0 || gx >= p.nx;
        if ((!oy || per_y) && (!ox || per_x)) {
          const int64_t g = int64_t(oy ? wrap(gy, p.ny) : gy) * p.nx + (ox ? wrap(gx, p.nx) : gx);
#pragma unroll
          for (int f = 0; f < NF; ++f) box[f * FB + br * W + bcol] = p.in[f][g];
        }
      };
      const int xs = cl + (W - cr);  // columns past the x sides, per row
      if (got && per_x && xs > 0)
        for (int c = tid; c < xs * BH; c += NCONS) {
          const int br = c / xs, k = c - br * xs;
          fix(br, k < cl ? k : cr + k - cl);
        }
      const int ys = rt + (BH - rb), inner = cr - cl;  // rows past the y sides
      if (got && per_y && ys > 0)
        for (int c = tid; c < ys * inner; c += NCONS) {
          const int k = c / inner, bcol = cl + (c - k * inner);
          fix(k < rt ? k : rb + k - rt, bcol);
        }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("bar.sync 1, %0;" ::"r"(NCONS) : "memory");
    }
    // u1 is the Dirichlet value 0 past a Dirichlet side, the computed
    // (periodic) value past a periodic one
    auto keep = [&](int tr, int tc) {
      const int gy = y0 + tr, gx = x0 + tc;
      const bool oy = gy < 0 || gy >= p.ny, ox = gx < 0 || gx >= p.nx;
      return (!oy || per_y) && (!ox || per_x);
    };
    auto sweep1 = [&](auto edge_tag) {
      constexpr bool EDGE = decltype(edge_tag)::value;
      F2 col[NF][NC];
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int k = 0; k < NC; ++k) col[f][k] = ld_pair(box + f * FB + (H - R + cy0 + k) * W + CW + cx2);
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        PairAcc<T, TX, TY, R, NF, NC> acc;
#pragma unroll
        for (int f = 0; f < NF; ++f) acc.b[f] = box + f * FB + (H + cy0 + r) * W + CW + cx2;
        acc.col = col;
        acc.r = r;
        acc.g = 0;
        F2 o[NF];
        F2 unused(0.f);
        p.op(acc, o, unused);
        const bool kp = !EDGE || keep(cy0 + r, cx2);
#pragma unroll
        for (int f = 0; f < NF; ++f)
          st_pair_f(u1 + f * FU + (R + cy0 + r) * W1 + 4 + cx2, kp ? stored_pair<T>(o[f]) : F2(0.f));
      }
      for (int c = tid; c < NRING; c += NCONS) {
        int tr, tc;
        if (c < 2 * R * 32) {  // the R rows above and below the tile
          const int row = c >> 5;
          tr = row < R ? row - R : TY + row - R;
          tc = (c & 31) * 2;
        } else if (c < 2 * R * 32 + 2 * TY) {  // the column pairs left and right of the tile
          const int d = c - 2 * R * 32;
          tr = d >> 1;
          tc = (d & 1) ? TX : -2;
        } else {  // box functions: those column pairs on the R rows above and below
          const int d = c - 2 * R * 32 - 2 * TY, row = d >> 1;
          tr = row < R ? row - R : TY + row - R;
          tc = (d & 1) ? TX : -2;
        }
        Smem2Acc<T, W, FB> acc{box + (H + tr) * W + CW + tc};
        F2 o[NF];
        F2 unused(0.f);
        p.op(acc, o, unused);
        const bool kp = !EDGE || keep(tr, tc);
#pragma unroll
        for (int f = 0; f < NF; ++f)
          st_pair_f(u1 + f * FU + (R + tr) * W1 + 4 + tc, kp ? stored_pair<T>(o[f]) : F2(0.f));
      }
    };
    if (got) {
      if (edge) sweep1(BoolTag<true>());
      else sweep1(BoolTag<false>());
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);  // the staged tile is no longer read
    }
    if (bar_or(1, NCONS, !got)) {  // u1 complete, or some warp gave up
      abort_flag = 1;
      break;
    }
    // ---- second sweep: the tile from u1
    {
      F2 col[NF][NC];
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int k = 0; k < NC; ++k) col[f][k] = ld_pair(u1 + f * FU + (cy0 + k) * W1 + 4 + cx2);
      const bool xin = x0 + cx2 < p.nx;
      const int64_t o_row = int64_t(y0 + cy0) * p.nx + x0 + cx2;
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        PairAcc<float, TX, TY, R, NF, NC> acc;
#pragma unroll
        for (int f = 0; f < NF; ++f) acc.b[f] = u1 + f * FU + (R + cy0 + r) * W1 + 4 + cx2;
        acc.col = col;
        acc.r = r;
        acc.g = 0;
        F2 o[NF];
        F2 unused(0.f);
        p.op(acc, o, unused);
        if (!edge || (xin && y0 + cy0 + r < p.ny)) {
#pragma unroll
          for (int f = 0; f < NF; ++f) st_pair(p.out[f] + o_row + int64_t(r) * p.nx, o[f]);
        }
      }
    }
  }
}

}  // namespace
}  // namespace lope
