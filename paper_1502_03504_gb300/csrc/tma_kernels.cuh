// Host-side runner of the TMA kernels: tile geometry, tensor maps, occupancy
// and launch (the kernels are in tma_device.cuh).  Included by k_tma.cu and
// k_tma_stage.cu.
#pragma once

#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "tma_device.cuh"

namespace lope {

namespace {

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}

template <class T> CUtensorMapDataType tma_dtype();
template <> CUtensorMapDataType tma_dtype<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> CUtensorMapDataType tma_dtype<double>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT64; }
template <> CUtensorMapDataType tma_dtype<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }

template <class T>
cudaError_t encode(CUtensorMap* m, const void* base, int rank, const int64_t* n /*x,y,z*/,
                   uint32_t bx, uint32_t by) {
  auto fn = get_encode();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[3] = {cuuint64_t(n[0]), cuuint64_t(n[1]), cuuint64_t(n[2])};
  cuuint64_t strides[2] = {cuuint64_t(n[0]) * sizeof(T), cuuint64_t(n[0] * n[1]) * sizeof(T)};
  cuuint32_t box[3] = {bx, by, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, tma_dtype<T>(), rank, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

constexpr int kZWaves = 3;
constexpr int kMinChunk = 48;

// Work split of the 3D z-march kernels: TX x TY tiles times z-chunks.  About
// kZWaves waves of blocks keep every resident slot busy (later blocks take the
// slots of blocks that finish early; edge tiles of periodic grids cost more
// per plane), but chunks stay at least kMinChunk planes long (each chunk
// stages its halo planes again); short grids get at most one wave (a few
// blocks past a full wave would double the time).
template <class P>
void zmarch_geometry(const Geom& g, P& p, int* blocks, int TX, int TY, int slots) {
  p.nx = int(g.n[2]);
  p.ny = int(g.n[1]);
  p.nz = int(g.n[0]);
  p.per_x = g.bc[2][0] == kPeriodic;
  p.per_y = g.bc[1][0] == kPeriodic;
  p.per_z = g.bc[0][0] == kPeriodic;
  p.tiles_x = (p.nx + TX - 1) / TX;
  p.tiles_y = (p.ny + TY - 1) / TY;
  const int ntiles = p.tiles_x * p.tiles_y;
  const int one_wave = std::max(1, slots / ntiles);
  int nzc = std::max(one_wave, std::min((kZWaves * slots) / ntiles, p.nz / kMinChunk));
  nzc = std::min(nzc, p.nz);
  p.zchunk = (p.nz + nzc - 1) / nzc;
  nzc = (p.nz + p.zchunk - 1) / p.zchunk;
  p.nunits = ntiles * nzc;
  *blocks = p.nunits;
}

// Tile shape, launch geometry and tensor maps of the TMA kernels for storage
// type T, rank RANK, halo radius R and NF fields; shared by the builtin
// runner below and by run-time compiled local functions (jit.cu).  PAIR:
// paired consumers (FP32/BF16 without reductions, radius <= 2).
// Tall or short tiles for this launch: lope_launch.tile_y 1 / 2 forces short /
// tall tiles on the TMA path; otherwise tall tiles from 2^22 points in 2D and
// 2^26 in 3D (a 512^3 grid), where enough tiles remain to fill every SM.
inline bool tma_tall(const StepArgs& a) {
  if (a.adjoint) return false;
  if (a.tile_y == 1) return false;
  if (a.tile_y == 2) return true;
  const int64_t n = a.g.n[0] * a.g.n[1] * a.g.n[2];
  return n >= (a.g.ndim == 3 ? (int64_t(1) << 26) : (int64_t(1) << 22));
}

template <class T, int RANK, int R, int NF, bool PAIR, bool TALL = true>
struct TmaShape {
  using Cfg = TmaCfg<T, RANK, R, NF, PAIR, TALL>;
  static constexpr int TX = Cfg::TX, TY = Cfg::TY, RY = Cfg::RY, S = Cfg::S;
  using L = Layout<T, TX, TY, R, NF>;
  static constexpr int THREADS = (PAIR ? TX / 2 : TX) * (TY / RY) + 32;
  static constexpr size_t SMEM = size_t(S) * L::STAGE_B + 2 * S * sizeof(uint64_t) + 128;
  static_assert(SMEM <= 227 * 1024, "stage ring exceeds the shared memory of a block");
  static_assert(THREADS <= 1024 && TY + 2 * R <= 256, "block or TMA box too large");

  // Fill the geometry fields of the kernel parameters and the block count;
  // occ(wrap) gives the resident blocks per SM of the kernel instance.
  template <class P, class Occ>
  static void geometry(const StepArgs& a, P& p, int* blocks, Occ&& occ) {
    const Geom& g = a.g;
    const bool wrap = g.bc[2][0] == kPeriodic || g.bc[1][0] == kPeriodic;
    const int slots = occ(wrap) * sm_count();
    if (RANK == 3) {
      zmarch_geometry(g, p, blocks, TX, TY, slots);
      return;
    }
    p.nx = int(g.n[2]);
    p.ny = int(g.n[1]);
    p.nz = int(g.n[0]);
    p.per_x = g.bc[2][0] == kPeriodic;
    p.per_y = g.bc[1][0] == kPeriodic;
    p.per_z = g.bc[0][0] == kPeriodic;
    p.tiles_x = (p.nx + TX - 1) / TX;
    p.tiles_y = (p.ny + TY - 1) / TY;
    p.nunits = p.tiles_x * p.tiles_y;
    p.zchunk = 1;
    *blocks = std::min(p.nunits, slots);
  }

  // Parameters common to every kernel instance (fields, flags) and the maps.
  // An external side of the slowest axis (z in 3D, y in 2D) extends the
  // tensor maps by R planes / rows of the caller's buffer beyond the grid:
  // there the halo is data, not the zero fill.
  template <class P>
  static cudaError_t prepare(const StepArgs& a, P& p, TmaMaps<NF>& maps) {
    for (int f = 0; f < NF; ++f) {
      p.in[f] = static_cast<const T*>(a.in[f]);
      p.out[f] = static_cast<T*>(a.out[f]);
    }
    p.partials = a.partials;
    p.err = a.err;
    const int sax = 3 - RANK;  // the slowest axis of the grid, in Geom order
    const int lo = a.g.bc[sax][0] == kExternal ? R : 0;
    const int hi = a.g.bc[sax][1] == kExternal ? R : 0;
    p.soff = lo;
    p.sext = (lo ? 1 : 0) | (hi ? 2 : 0);
    int64_t n[3] = {a.g.n[2], a.g.n[1], a.g.n[0]};
    n[RANK - 1] += lo + hi;
    const int64_t before = int64_t(lo) * (RANK == 3 ? a.g.n[2] * a.g.n[1] : a.g.n[2]);
    // box functions stage the wrapped halo columns of the halo rows too
    const uint32_t colh = a.s.star ? TY : TY + 2 * R;
    for (int f = 0; f < NF; ++f) {
      const T* base = static_cast<const T*>(a.in[f]) - before;
      cudaError_t e;
      if ((e = encode<T>(&maps.wide[f], base, RANK, n, L::W, TY + 2 * R)) ||
          (e = encode<T>(&maps.rows[f], base, RANK, n, L::W, R)) ||
          (e = encode<T>(&maps.cols[f], base, RANK, n, L::CW, colh)))
        return e;
    }
    return cudaSuccess;
  }
};

// The two-sweep z-march (tma3d_tb2_kernel): 64 x TY tiles of paired
// consumers, RY = 8 rows per warp, an S-stage ring of input planes staged
// with a 2-row halo, and three u1 slots per warp.
template <class T, int TY_, int S_>
struct Tb2Shape {
  static constexpr int TX = 64, TY = TY_, RY = 8, S = S_, H = 2;
  using L = Layout<T, TX, TY, H, 1>;
  using SL = Tb2Slots<TX, TY, RY>;
  static constexpr int THREADS = 32 * SL::NW + 32;
  static constexpr size_t SMEM = size_t(S) * L::OFF_COLL + SL::BYTES + 2 * S * sizeof(uint64_t) + 128;
  static_assert(SMEM <= 227 * 1024, "two-sweep ring exceeds the shared memory of a block");

  template <class P>
  static cudaError_t prepare(const StepArgs& a, P& p, TmaMaps<1>& maps) {
    p.in[0] = static_cast<const T*>(a.in[0]);
    p.out[0] = static_cast<T*>(a.out[0]);
    p.partials = nullptr;
    p.err = a.err;
    p.soff = 0;
    p.sext = 0;
    const int64_t n[3] = {a.g.n[2], a.g.n[1], a.g.n[0]};
    return encode<T>(&maps.wide[0], a.in[0], 3, n, L::W, TY + 2 * H);
  }
};

// The two-sweep 2D tiles (tma2d_tb2_kernel): 64 x TY tiles of paired
// consumers, RY rows per warp, a 3-stage ring of tiles staged with a 2R-row
// halo, and two u1 buffers per field.  One field: 128-row tiles; several: 32
// rows (the ring and the u1 buffers of three fields fit 227 KB at that height).
template <class T, int R, int RY_ = 8, int NF = 1>
struct Tb2Shape2D {
  static constexpr int TX = 64, TY = NF == 1 ? 128 : 32, RY = RY_, S = 3, H = 2 * R;
  using L = Layout<T, TX, TY, H, NF>;
  using M = Tb2Mem2D<T, TY, R, NF>;
  static constexpr int THREADS = 32 * (TY / RY) + 32;
  static constexpr size_t U1B = M::U1B;
  static constexpr size_t SMEM =
      size_t(S) * M::STAGE + 2 * NF * U1B + 2 * S * sizeof(uint64_t) + 128;
  static_assert(SMEM <= 227 * 1024, "two-sweep tiles exceed the shared memory of a block");

  template <class P>
  static cudaError_t prepare(const StepArgs& a, P& p, TmaMaps<NF>& maps) {
    const int64_t n[3] = {a.g.n[2], a.g.n[1], a.g.n[0]};
    for (int f = 0; f < NF; ++f) {
      p.in[f] = static_cast<const T*>(a.in[f]);
      p.out[f] = static_cast<T*>(a.out[f]);
      cudaError_t e = encode<T>(&maps.wide[f], a.in[f], 2, n, L::W, TY + 2 * H);
      if (e != cudaSuccess) return e;
    }
    p.partials = nullptr;
    p.err = a.err;
    p.soff = 0;
    p.sext = 0;
    return cudaSuccess;
  }
};

// The two-sweep z-march with block-shared u1 planes (tma3d_tb2s_kernel): 64 x
// 64 tiles, 16 consumer warps of 4 rows, a 6-stage ring of input planes
// staged with a 2-row halo, three shared u1 planes.
template <class T>
struct Tb2sShape {
  static constexpr int TX = 64, TY = 64, RY = 4, S = 6, H = 2;
  using L = Layout<T, TX, TY, H, 1>;
  static constexpr int THREADS = 32 * (TY / RY) + 32;
  static constexpr size_t SMEM = size_t(S) * L::OFF_COLL + 3 * size_t(TY + 2) * (TX + 8) * 4 +
                                 2 * S * sizeof(uint64_t) + 128;
  static_assert(SMEM <= 227 * 1024, "two-sweep ring exceeds the shared memory of a block");

  template <class P>
  static cudaError_t prepare(const StepArgs& a, P& p, TmaMaps<1>& maps) {
    p.in[0] = static_cast<const T*>(a.in[0]);
    p.out[0] = static_cast<T*>(a.out[0]);
    p.partials = nullptr;
    p.err = a.err;
    p.soff = 0;
    p.sext = 0;
    const int64_t n[3] = {a.g.n[2], a.g.n[1], a.g.n[0]};
    return encode<T>(&maps.wide[0], a.in[0], 3, n, L::W, TY + 2 * H);
  }
};

// Geometry of the two-sweep 2D tiles (persistent blocks over the tile list).
template <class Sh2, class P>
int tb2_2d_geometry(const Geom& g, P& p, int occ) {
  p.nx = int(g.n[2]);
  p.ny = int(g.n[1]);
  p.nz = 1;
  p.per_x = g.bc[2][0] == kPeriodic;
  p.per_y = g.bc[1][0] == kPeriodic;
  p.per_z = 0;
  p.tiles_x = (p.nx + Sh2::TX - 1) / Sh2::TX;
  p.tiles_y = (p.ny + Sh2::TY - 1) / Sh2::TY;
  p.nunits = p.tiles_x * p.tiles_y;
  p.zchunk = 1;
  return std::min(p.nunits, occ * sm_count());
}

// Whether the two-sweep kernels run this launch: in 3D a radius-1 star
// function of one field (diffusion builtin, linear table or run-time compiled
// function); in 2D a radius-1 or 2 function, star or box, of one to three
// fields (jacobi5, star9r2, the shallow-water builtins, linear tables,
// run-time compiled functions); FP32 or BF16 storage, no external
// halo, Dirichlet sides of value 0, no adjoint, no multi-stage combination.
// The 3D z-march also needs every x and y side Dirichlet (its ring of u1 is
// masked, not wrapped); the 2D tiles take periodic sides too.
inline bool tb2_supported(const StepArgs& a) {
  const Geom& g = a.g;
  const StencilDesc& s = a.s;
  if ((g.nf != 1 && (g.ndim != 2 || (s.kind != kSwe && s.kind != kSweFlux && s.kind != kUser))) ||
      (!s.star && g.ndim != 2) || a.adjoint || a.stage >= 2)
    return false;
  if (g.dtype != kF32 && g.dtype != kBF16) return false;
  for (int ax = 0; ax < 3; ++ax)
    for (int sd = 0; sd < 2; ++sd)
      if (g.bc[ax][sd] == kExternal || (g.bc[ax][sd] == kDirichlet && g.bval[ax][sd] != 0.0))
        return false;
  if (g.ndim == 3) {
    if (s.radius != 1 || (s.kind != kDiff7 && s.kind != kLinear && s.kind != kUser)) return false;
    for (int ax = 1; ax < 3; ++ax)
      for (int sd = 0; sd < 2; ++sd)
        if (g.bc[ax][sd] != kDirichlet) return false;
    return true;
  }
  return s.radius <= 2 && (s.kind == kJacobi5 || s.kind == kStar9r2 || s.kind == kLinear ||
                            s.kind == kUser || s.kind == kSwe || s.kind == kSweFlux);
}

// Paired consumers for FP32/BF16 storage (radius <= 2), adjoint functors
// included: their per-point reduction is summed per lane (tile2d_pair /
// march3d_pair).  Adjoint launches take the short tiles (tma_tall), where the
// paired adjoint does not spill: forward + adjoint of a 256^3 grid measured
// 9.75 ms against 11.6 ms on single-column consumers.
template <class T, int R>
constexpr bool tma_pair(bool reduces) {
  (void)reduces;
  return !std::is_same<T, double>::value && R <= 2 && TmaTx<T>::TX == 64;
}

template <class Op, class T, int RANK>
struct TmaRunner {
  static constexpr bool PAIR = tma_pair<T, Op::R>(Op::REDUCES);
  template <bool TALL> using Sh = TmaShape<T, RANK, Op::R, Op::NF, PAIR, TALL>;

  template <bool TALL, bool WRAP> static auto kernel_w() {
    using S_ = Sh<TALL>;
    if constexpr (RANK == 2) return &tma2d_kernel<Op, T, S_::TX, S_::TY, S_::RY, S_::S, WRAP, PAIR>;
    else return &tma3d_kernel<Op, T, S_::TX, S_::TY, S_::RY, S_::S, WRAP, PAIR>;
  }

  template <bool TALL, bool WRAP> static int occupancy_w() {
    static int occ = -1;
    if (occ < 0) {
      cudaFuncSetAttribute(kernel_w<TALL, WRAP>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(Sh<TALL>::SMEM));
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel_w<TALL, WRAP>(), Sh<TALL>::THREADS,
                                                        Sh<TALL>::SMEM) != cudaSuccess)
        o = 1;
      occ = o > 0 ? o : 1;
    }
    return occ;
  }
  template <bool TALL> static int occupancy(bool wrap) {
    return wrap ? occupancy_w<TALL, true>() : occupancy_w<TALL, false>();
  }

  template <class P>
  static void geometry(const StepArgs& a, P& p, int* blocks) {
    if (tma_tall(a)) Sh<true>::geometry(a, p, blocks, [](bool w) { return occupancy<true>(w); });
    else Sh<false>::geometry(a, p, blocks, [](bool w) { return occupancy<false>(w); });
  }

  template <bool TALL>
  static cudaError_t run_t(const StepArgs& a, const Op& op, int* blocks_out) {
    using S_ = Sh<TALL>;
    TmaParams<Op, T> p;
    p.op = op;
    int blocks = 0;
    S_::geometry(a, p, &blocks, [](bool w) { return occupancy<TALL>(w); });
    if (blocks_out) *blocks_out = blocks;
    if (Op::REDUCES && (!a.partials || blocks > a.partial_count)) return cudaErrorInvalidValue;
    TmaMaps<Op::NF> maps;
    cudaError_t e = S_::prepare(a, p, maps);
    if (e != cudaSuccess) return e;
    if (p.per_x || p.per_y)
      kernel_w<TALL, true>()<<<blocks, S_::THREADS, S_::SMEM, a.stream>>>(maps, p);
    else
      kernel_w<TALL, false>()<<<blocks, S_::THREADS, S_::SMEM, a.stream>>>(maps, p);
    count_launches(1);
    return cudaGetLastError();
  }

  static cudaError_t run(const StepArgs& a, const Op& op, int* blocks_out) {
    return tma_tall(a) ? run_t<true>(a, op, blocks_out) : run_t<false>(a, op, blocks_out);
  }

  // Two sweeps in one launch (3D radius-1 star functions of one field; see
  // tb2_supported).  lope_launch.tile_y 1 / 2 forces 32- / 64-row tiles.
  template <int TY, int S>
  static cudaError_t run_tb2_t(const StepArgs& a, const Op& op, int* blocks_out) {
    if constexpr (RANK == 3 && Op::R == 1 && Op::NF == 1 && Op::STAR && PAIR && !Op::REDUCES) {
      using Sh2 = Tb2Shape<T, TY, S>;
      auto kern = &tma3d_tb2_kernel<Op, T, Sh2::TX, Sh2::TY, Sh2::RY, Sh2::S>;
      static int occ = -1;
      if (occ < 0) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh2::SMEM));
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, Sh2::THREADS, Sh2::SMEM) !=
            cudaSuccess)
          o = 1;
        occ = o > 0 ? o : 1;
      }
      TmaParams<Op, T> p;
      p.op = op;
      int blocks = 0;
      zmarch_geometry(a.g, p, &blocks, Sh2::TX, Sh2::TY, occ * sm_count());
      if (blocks_out) *blocks_out = blocks;
      TmaMaps<1> maps;
      cudaError_t e = Sh2::prepare(a, p, maps);
      if (e != cudaSuccess) return e;
      kern<<<blocks, Sh2::THREADS, Sh2::SMEM, a.stream>>>(maps, p);
      count_launches(1);
      return cudaGetLastError();
    } else {
      (void)a;
      (void)op;
      (void)blocks_out;
      return cudaErrorNotSupported;
    }
  }

  template <bool WRAP, int RY>
  static cudaError_t run_tb2_2d_t(const StepArgs& a, const Op& op, int* blocks_out) {
    if constexpr (RANK == 2 && Op::R <= 2 && PAIR && !Op::REDUCES) {
      using Sh2 = Tb2Shape2D<T, Op::R, RY, Op::NF>;
      auto kern = &tma2d_tb2_kernel<Op, T, Sh2::TY, Sh2::RY, Sh2::S, WRAP>;
      static int occ = -1;
      if (occ < 0) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh2::SMEM));
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, Sh2::THREADS, Sh2::SMEM) !=
            cudaSuccess)
          o = 1;
        occ = o > 0 ? o : 1;
      }
      TmaParams<Op, T> p;
      p.op = op;
      const int blocks = tb2_2d_geometry<Sh2>(a.g, p, occ);
      if (blocks_out) *blocks_out = blocks;
      TmaMaps<Op::NF> maps;
      cudaError_t e = Sh2::prepare(a, p, maps);
      if (e != cudaSuccess) return e;
      kern<<<blocks, Sh2::THREADS, Sh2::SMEM, a.stream>>>(maps, p);
      count_launches(1);
      return cudaGetLastError();
    } else {
      (void)a;
      (void)op;
      (void)blocks_out;
      return cudaErrorNotSupported;
    }
  }

  // The two-sweep march with block-shared u1 planes: 64 x 64 tiles, 16
  // consumer warps of 4 rows.
  static cudaError_t run_tb2s(const StepArgs& a, const Op& op, int* blocks_out) {
    if constexpr (RANK == 3 && Op::R == 1 && Op::NF == 1 && Op::STAR && PAIR && !Op::REDUCES) {
      using Sh = Tb2sShape<T>;
      constexpr int TX = Sh::TX, TY = Sh::TY, THREADS = Sh::THREADS;
      constexpr size_t SMEM = Sh::SMEM;
      auto kern = &tma3d_tb2s_kernel<Op, T, TX, TY, Sh::RY, Sh::S>;
      static int occ = -1;
      if (occ < 0) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM));
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, THREADS, SMEM) != cudaSuccess) o = 1;
        occ = o > 0 ? o : 1;
      }
      TmaParams<Op, T> p;
      p.op = op;
      int blocks = 0;
      zmarch_geometry(a.g, p, &blocks, TX, TY, occ * sm_count());
      if (blocks_out) *blocks_out = blocks;
      TmaMaps<1> maps;
      cudaError_t e = Sh::prepare(a, p, maps);
      if (e != cudaSuccess) return e;
      kern<<<blocks, THREADS, SMEM, a.stream>>>(maps, p);
      count_launches(1);
      return cudaGetLastError();
    } else {
      (void)a;
      (void)op;
      (void)blocks_out;
      return cudaErrorNotSupported;
    }
  }

  static cudaError_t run_tb2(const StepArgs& a, const Op& op, int* blocks_out) {
    if constexpr (RANK == 3) {
      // Block-shared u1 planes (16 warps) unless lope_launch.tile_y 1 / 2
      // asks for the per-warp slots on 32- / 64-row tiles (8 warps).  The
      // shared planes measured faster at every size: diff7 FP32 512^3, 50
      // sweeps: 5.46 ms against 5.91 ms.
      if (a.tile_y != 1 && a.tile_y != 2) return run_tb2s(a, op, blocks_out);
    }
    if constexpr (RANK == 2) {
      // One field: lope_launch.tile_y 1 takes 16 rows per consumer warp (8
      // warps), else 8 rows (16 warps).  Several fields (32-row tiles): star
      // functions 2 rows (16 warps; linear shallow water 4096^2 x200 BF16
      // periodic 7.18 against 7.57 ms with 4 rows, FP32 equal), box
      // functions 4 rows (8 warps; nonlinear shallow water FP32 56.4
      // against 58.4 us per sweep); tile_y 1 takes the other layout.
      const bool wrap = a.g.bc[2][0] == kPeriodic || a.g.bc[1][0] == kPeriodic;
      constexpr int RY_M = Op::STAR ? 2 : 4, RY_N = Op::STAR ? 4 : 2;
      constexpr int RY_A = Op::NF == 1 ? 16 : RY_N, RY_B = Op::NF == 1 ? 8 : RY_M;
      if (a.tile_y == 1)
        return wrap ? run_tb2_2d_t<true, RY_A>(a, op, blocks_out)
                    : run_tb2_2d_t<false, RY_A>(a, op, blocks_out);
      return wrap ? run_tb2_2d_t<true, RY_B>(a, op, blocks_out)
                  : run_tb2_2d_t<false, RY_B>(a, op, blocks_out);
    }
    if (a.tile_y == 1) return run_tb2_t<32, 6>(a, op, blocks_out);
    return run_tb2_t<64, 6>(a, op, blocks_out);
  }
};

// The z-march with planes copied by producer warps (ca3d_kernel), for FP32 /
// FP64 3D grids whose rows TMA cannot stage: 64 x 64 tiles (32 x 32 for FP64;
// lope_launch.tile_y 1 forces 64 x 32 / 32 x 32), sixteen producer warps (eight
// for FP64, whose rows take half the copies), as many planes in flight as 227
// KB of shared memory hold (at most kCaMaxStages), and z chunks sized in whole
// waves of the measured occupancy.
template <class T> constexpr int ca_producer_warps() { return sizeof(T) == 8 ? 8 : 16; }
constexpr int kCaMaxStages = 12;

template <class Op, class T>
struct CaRunner {
  static constexpr bool PAIR = tma_pair<T, Op::R>(Op::REDUCES);
  static constexpr int NPW = ca_producer_warps<T>();
  template <bool TALL> using Sh = TmaShape<T, 3, Op::R, Op::NF, PAIR, TALL>;
  template <bool TALL> using Lay = typename Sh<TALL>::L;
  template <bool TALL> static constexpr int stages() {
    constexpr int fit = int((227 * 1024 - 1024) / Lay<TALL>::STAGE_B);
    return fit < kCaMaxStages ? fit : kCaMaxStages;
  }
  template <bool TALL> static constexpr size_t smem() {
    return size_t(stages<TALL>()) * Lay<TALL>::STAGE_B + 2 * stages<TALL>() * sizeof(uint64_t) + 128;
  }
  template <bool TALL> static auto kernel() {
    using S_ = Sh<TALL>;
    static_assert(stages<TALL>() >= Op::R + 2 && smem<TALL>() <= 227 * 1024, "stage ring");
    return &ca3d_kernel<Op, T, S_::TX, S_::TY, S_::RY, stages<TALL>(), PAIR, NPW>;
  }
  template <bool TALL> static constexpr int threads() {
    return Sh<TALL>::THREADS - 32 + 32 * NPW;
  }
  template <bool TALL> static int occupancy() {
    static int occ = -1;
    if (occ < 0) {
      cudaFuncSetAttribute(kernel<TALL>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(smem<TALL>()));
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel<TALL>(), threads<TALL>(),
                                                        smem<TALL>()) != cudaSuccess)
        o = 1;
      occ = o > 0 ? o : 1;
    }
    return occ;
  }
  template <bool TALL>
  static cudaError_t run_t(const StepArgs& a, const Op& op, int zchunk, int blocks) {
    using S_ = Sh<TALL>;
    TmaParams<Op, T> p;
    p.op = op;
    p.nx = int(a.g.n[2]);
    p.ny = int(a.g.n[1]);
    p.nz = int(a.g.n[0]);
    p.per_x = p.per_y = p.per_z = 0;  // the producers apply every side's rule
    p.tiles_x = (p.nx + S_::TX - 1) / S_::TX;
    p.tiles_y = (p.ny + S_::TY - 1) / S_::TY;
    p.zchunk = zchunk;
    p.nunits = blocks;
    p.soff = 0;
    p.sext = 0;
    for (int f = 0; f < Op::NF; ++f) {
      p.in[f] = static_cast<const T*>(a.in[f]);
      p.out[f] = static_cast<T*>(a.out[f]);
    }
    p.partials = a.partials;
    p.err = a.err;
    if (Op::REDUCES && (!a.partials || blocks > a.partial_count)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kernel<TALL>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem<TALL>()));
    if (e != cudaSuccess) return e;
    kernel<TALL>()<<<blocks, threads<TALL>(), smem<TALL>(), a.stream>>>(a.g, p);
    count_launches(1);
    return cudaGetLastError();
  }
  // chunks(tx, ty, per_sm, &blocks, &zchunk): the z-chunk split of the caller.
  // Tall tiles unless lope_launch.tile_y is 1 (measured: diff7 FP32
  // 130 x 500 x 510, 76 against 123 us per sweep; 511^3, 272 against 454 us).
  template <class Chunks>
  static cudaError_t run(const StepArgs& a, const Op& op, Chunks&& chunks) {
    int blocks = 0, zchunk = 0;
    if (a.tile_y != 1) {
      if (!chunks(Sh<true>::TX, Sh<true>::TY, occupancy<true>(), &blocks, &zchunk))
        return cudaErrorInvalidConfiguration;
      return run_t<true>(a, op, zchunk, blocks);
    }
    if (!chunks(Sh<false>::TX, Sh<false>::TY, occupancy<false>(), &blocks, &zchunk))
      return cudaErrorInvalidConfiguration;
    return run_t<false>(a, op, zchunk, blocks);
  }
};

}  // namespace
}  // namespace lope
