// TMA-staged stencil kernels for star-shaped local functions.
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
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "device_common.cuh"

namespace lope {

namespace {

constexpr int kTy = 32;  // tile rows
constexpr int kRy = 8;   // rows per consumer thread

template <class T> struct TmaCfg;
template <> struct TmaCfg<float> { static constexpr int TX = 64, S2 = 4, S3 = 6; };
template <> struct TmaCfg<double> { static constexpr int TX = 32, S2 = 4, S3 = 6; };
template <> struct TmaCfg<__nv_bfloat16> { static constexpr int TX = 64, S2 = 4, S3 = 6; };

template <int NF> struct TmaMaps {
  CUtensorMap main[NF];  // box {TX, TY+2R[, 1]}
  CUtensorMap body[NF];  // box {TX, TY[, 1]}
  CUtensorMap row[NF];   // box {TX, 1[, 1]}
  CUtensorMap cols[NF];  // box {CW, TY[, 1]}
};

template <class Op, class T> struct TmaParams {
  Op op;
  T* out[kMaxFields];
  int nx, ny, nz;
  int per_x, per_y, per_z;
  int tiles_x, tiles_y;
  int zchunk;     // 3D: output planes per unit
  int nunits;     // number of work units
  double* partials;
  int* err;
};

template <class T, int TX, int R, int NF> struct Layout {
  static constexpr int CW = 16 / int(sizeof(T));
  static constexpr uint32_t MAIN_B = (kTy + 2 * R) * TX * sizeof(T);
  static constexpr uint32_t MAIN_BA = (MAIN_B + 127) / 128 * 128;
  static constexpr uint32_t SLOT_B = kTy * CW * sizeof(T);
  static constexpr uint32_t SLOT_BA = (SLOT_B + 127) / 128 * 128;
  static constexpr uint32_t FIELD_B = MAIN_BA + 2 * SLOT_BA;
  static constexpr uint32_t STAGE_B = NF * FIELD_B;
  static constexpr uint32_t TX_BYTES = NF * (MAIN_B + 2 * SLOT_B);
};

// Accessor over one staged plane/tile.  (cx, cy) is the local element inside
// the tile, already clamped into the valid region; nvx/nvy are the valid
// extents of this (possibly ragged) tile.  In 3D, z offsets come from the
// caller's register queue q[field][R + dz].
template <class T, int TX, int R, int NF, int NQ>
struct PlaneAcc {
  using L = Layout<T, TX, R, NF>;
  using C = C_t<T>;
  const unsigned char* stage;
  int cx, cy, nvx, nvy;
  int64_t g;
  const C (*q)[NQ];  // NQ = 2R+1 in 3D, 1 in 2D (unused)

  __device__ __forceinline__ const T* mainp(int f) const {
    return reinterpret_cast<const T*>(stage + f * L::FIELD_B);
  }
  __device__ __forceinline__ C operator()(int f, int dx, int dy, int dz) const {
    if (dz != 0) return q[f][R + dz];
    const T* m = mainp(f);
    if (dx != 0) {
      int col = cx + dx;
      if (col < 0) {
        const T* left = reinterpret_cast<const T*>(stage + f * L::FIELD_B + L::MAIN_BA);
        return to_c(left[cy * L::CW + L::CW + col]);
      }
      if (col >= nvx) {
        const T* right =
            reinterpret_cast<const T*>(stage + f * L::FIELD_B + L::MAIN_BA + L::SLOT_BA);
        return to_c(right[cy * L::CW + (col - nvx)]);
      }
      return to_c(m[(R + cy) * TX + col]);
    }
    if (dy != 0) {
      int row = cy + dy;
      int rr = row >= nvy ? R + kTy + (row - nvy) : R + row;
      return to_c(m[rr * TX + cx]);
    }
    if (NQ > 1) return q[f][R];
    return to_c(m[(R + cy) * TX + cx]);
  }
  __device__ __forceinline__ int64_t gidx() const { return g; }
};

// Issue the copies of one tile/plane of every field into stage `st`.
template <class T, int TX, int R, int NF, int RANK>
__device__ __forceinline__ void issue_plane(const TmaMaps<NF>& maps, unsigned char* st,
                                            uint64_t* bar, int x0, int y0, int nvx, int nvy,
                                            int z, int nx, int ny, int per_x, int per_y) {
  using L = Layout<T, TX, R, NF>;
  mbar_arrive_expect_tx(bar, L::TX_BYTES);
  const bool yedge = per_y && (y0 < R || y0 + kTy + R > ny);
  const int xl = per_x ? wrap(x0 - L::CW, nx) : x0 - L::CW;
  const int xr = per_x ? wrap(x0 + nvx, nx) : x0 + nvx;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    unsigned char* m = st + f * L::FIELD_B;
    unsigned char* left = m + L::MAIN_BA;
    unsigned char* right = left + L::SLOT_BA;
    if (!yedge) {
      if (RANK == 2) tma_load_2d(m, &maps.main[f], x0, y0 - R, bar);
      else tma_load_3d(m, &maps.main[f], x0, y0 - R, z, bar);
    } else {
      unsigned char* body = m + R * TX * sizeof(T);
      if (RANK == 2) tma_load_2d(body, &maps.body[f], x0, y0, bar);
      else tma_load_3d(body, &maps.body[f], x0, y0, z, bar);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        unsigned char* lo = m + j * TX * sizeof(T);
        unsigned char* hi = m + (R + kTy + j) * TX * sizeof(T);
        int ylo = wrap(y0 - R + j, ny), yhi = wrap(y0 + nvy + j, ny);
        if (RANK == 2) {
          tma_load_2d(lo, &maps.row[f], x0, ylo, bar);
          tma_load_2d(hi, &maps.row[f], x0, yhi, bar);
        } else {
          tma_load_3d(lo, &maps.row[f], x0, ylo, z, bar);
          tma_load_3d(hi, &maps.row[f], x0, yhi, z, bar);
        }
      }
    }
    if (RANK == 2) {
      tma_load_2d(left, &maps.cols[f], xl, y0, bar);
      tma_load_2d(right, &maps.cols[f], xr, y0, bar);
    } else {
      tma_load_3d(left, &maps.cols[f], xl, y0, z, bar);
      tma_load_3d(right, &maps.cols[f], xr, y0, z, bar);
    }
  }
}

__device__ __forceinline__ unsigned char* align128(unsigned char* p) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 127) &
                                          ~uintptr_t(127));
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

// ------------------------------------------------------------------ 2D tiles
template <class Op, class T, int TX, int S>
__global__ void __launch_bounds__(TX * (kTy / kRy) + 32)
    tma2d_kernel(const __grid_constant__ TmaMaps<Op::NF> maps, const TmaParams<Op, T> p) {
  using C = C_t<T>;
  constexpr int R = Op::R, NF = Op::NF;
  using L = Layout<T, TX, R, NF>;
  constexpr int NCONS = TX * (kTy / kRy);
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
      for (int f = 0; f < NF; ++f) {
        tma_prefetch_desc(&maps.main[f]);
        tma_prefetch_desc(&maps.cols[f]);
      }
      int i = 0;
      for (int t = blockIdx.x; t < p.nunits; t += gridDim.x, ++i) {
        const int s = i % S;
        const uint32_t ph = (i / S) & 1;
        if (i >= S && !mbar_wait_bounded(&empty[s], ph ^ 1, p.err)) {
          abort_flag = 1;
          break;
        }
        if (abort_flag) break;
        const int x0 = (t % p.tiles_x) * TX, y0 = (t / p.tiles_x) * kTy;
        const int nvx = min(TX, p.nx - x0), nvy = min(kTy, p.ny - y0);
        issue_plane<T, TX, R, NF, 2>(maps, smem + s * L::STAGE_B, &full[s], x0, y0, nvx, nvy, 0,
                                     p.nx, p.ny, p.per_x, p.per_y);
      }
      if (abort_flag) {  // let copies already issued land before the block exits
        for (int k = max(0, i - S); k < i; ++k) mbar_wait_bounded(&full[k % S], (k / S) & 1, nullptr);
      }
    }
    return;
  }

  const int cx_t = tid % TX, cy0 = (tid / TX) * kRy, lane = tid % 32;
  double red = 0.0;
  int i = 0;
  for (int t = blockIdx.x; t < p.nunits; t += gridDim.x, ++i) {
    const int s = i % S;
    if (!mbar_wait_bounded(&full[s], (i / S) & 1, p.err) || abort_flag) {
      abort_flag = 1;
      break;
    }
    const int x0 = (t % p.tiles_x) * TX, y0 = (t / p.tiles_x) * kTy;
    const int nvx = min(TX, p.nx - x0), nvy = min(kTy, p.ny - y0);
    PlaneAcc<T, TX, R, NF, 1> acc;
    acc.stage = smem + s * L::STAGE_B;
    acc.nvx = nvx;
    acc.nvy = nvy;
    acc.cx = min(cx_t, nvx - 1);
    acc.q = nullptr;
#pragma unroll
    for (int r = 0; r < kRy; ++r) {
      const int cy_t = cy0 + r;
      acc.cy = min(cy_t, nvy - 1);
      const bool valid = cx_t < nvx && cy_t < nvy;
      const int64_t gi = int64_t(y0 + acc.cy) * p.nx + x0 + acc.cx;
      acc.g = gi;
      C o[NF];
      double r1 = 0.0;
      p.op(acc, o, r1);
      if (valid) {
#pragma unroll
        for (int f = 0; f < NF; ++f) p.out[f][gi] = from_c<T>(o[f]);
        red += r1;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  if (Op::REDUCES) block_accumulate<NCONS>(red, p.partials, red_scratch);
}

// ------------------------------------------------------------------ 3D z-march
template <class Op, class T, int TX, int S>
__global__ void __launch_bounds__(TX * (kTy / kRy) + 32, 2)
    tma3d_kernel(const __grid_constant__ TmaMaps<Op::NF> maps, const TmaParams<Op, T> p) {
  using C = C_t<T>;
  constexpr int R = Op::R, NF = Op::NF, NQ = 2 * R + 1;
  using L = Layout<T, TX, R, NF>;
  constexpr int NCONS = TX * (kTy / kRy);
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
  const int x0 = (tile % p.tiles_x) * TX, y0 = (tile / p.tiles_x) * kTy;
  const int nvx = min(TX, p.nx - x0), nvy = min(kTy, p.ny - y0);
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
      for (int f = 0; f < NF; ++f) {
        tma_prefetch_desc(&maps.main[f]);
        tma_prefetch_desc(&maps.cols[f]);
      }
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
        issue_plane<T, TX, R, NF, 3>(maps, smem + s * L::STAGE_B, &full[s], x0, y0, nvx, nvy, z,
                                     p.nx, p.ny, p.per_x, p.per_y);
      }
      if (abort_flag) {
        for (int k = max(0, j - S); k < j; ++k) mbar_wait_bounded(&full[k % S], (k / S) & 1, nullptr);
      }
    }
    return;
  }

  const int cx_t = tid % TX, cy0 = (tid / TX) * kRy, lane = tid % 32;
  const int cx = min(cx_t, nvx - 1);
  C q[kRy][NF][NQ];
  double red = 0.0;
  bool ok = true;

  auto release = [&](int j) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[j % S]);
  };
  // Load the centre values of staged plane j into the top of each queue.
  auto shift_in = [&](int j) -> bool {
    const int s = j % S;
    if (!mbar_wait_bounded(&full[s], (j / S) & 1, p.err) || abort_flag) {
      abort_flag = 1;
      return false;
    }
    const T* st = reinterpret_cast<const T*>(smem + s * L::STAGE_B);
#pragma unroll
    for (int r = 0; r < kRy; ++r) {
      const int cy = min(cy0 + r, nvy - 1);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
#pragma unroll
        for (int k = 0; k < NQ - 1; ++k) q[r][f][k] = q[r][f][k + 1];
        q[r][f][NQ - 1] =
            to_c(reinterpret_cast<const T*>(reinterpret_cast<const unsigned char*>(st) +
                                            f * L::FIELD_B)[(R + cy) * TX + cx]);
      }
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
    PlaneAcc<T, TX, R, NF, NQ> acc;
    acc.stage = smem + (jc % S) * L::STAGE_B;
    acc.nvx = nvx;
    acc.nvy = nvy;
    acc.cx = cx;
    const int z = z0 + m;
#pragma unroll
    for (int r = 0; r < kRy; ++r) {
      const int cy_t = cy0 + r;
      acc.cy = min(cy_t, nvy - 1);
      acc.q = q[r];
      const bool valid = cx_t < nvx && cy_t < nvy;
      const int64_t gi = (int64_t(z) * p.ny + (y0 + acc.cy)) * p.nx + x0 + cx;
      acc.g = gi;
      C o[NF];
      double r1 = 0.0;
      p.op(acc, o, r1);
      if (valid) {
#pragma unroll
        for (int f = 0; f < NF; ++f) p.out[f][gi] = from_c<T>(o[f]);
        red += r1;
      }
    }
    release(jc);
    if (jn >= np - R) release(jn);  // above z1-1: centres only
  }
  if (Op::REDUCES) block_accumulate<NCONS>(red, p.partials, red_scratch);
}

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

template <class Op, class T, int RANK>
struct TmaRunner {
  static constexpr int TX = TmaCfg<T>::TX;
  static constexpr int S = RANK == 2 ? TmaCfg<T>::S2 : TmaCfg<T>::S3;
  using L = Layout<T, TX, Op::R, Op::NF>;
  static constexpr int THREADS = TX * (kTy / kRy) + 32;
  static constexpr size_t SMEM = size_t(S) * L::STAGE_B + 2 * S * sizeof(uint64_t) + 128;

  static auto kernel() {
    if constexpr (RANK == 2) return &tma2d_kernel<Op, T, TX, S>;
    else return &tma3d_kernel<Op, T, TX, S>;
  }

  static int occupancy() {
    static int occ = -1;
    if (occ < 0) {
      cudaFuncSetAttribute(kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM));
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel(), THREADS, SMEM) !=
          cudaSuccess)
        o = 1;
      occ = o > 0 ? o : 1;
    }
    return occ;
  }

  template <class P>
  static void geometry(const StepArgs& a, P& p, int* blocks) {
    const Geom& g = a.g;
    p.nx = int(g.n[2]);
    p.ny = int(g.n[1]);
    p.nz = int(g.n[0]);
    p.per_x = g.bc[2][0] == kPeriodic;
    p.per_y = g.bc[1][0] == kPeriodic;
    p.per_z = g.bc[0][0] == kPeriodic;
    p.tiles_x = (p.nx + TX - 1) / TX;
    p.tiles_y = (p.ny + kTy - 1) / kTy;
    const int ntiles = p.tiles_x * p.tiles_y;
    const int slots = occupancy() * sm_count();
    if (RANK == 2) {
      p.nunits = ntiles;
      p.zchunk = 1;
      *blocks = std::min(ntiles, slots);
    } else {
      // Split z so that the blocks fill the resident slots once.
      int nzc = std::max(1, slots / ntiles);
      nzc = std::min(nzc, p.nz);
      p.zchunk = (p.nz + nzc - 1) / nzc;
      nzc = (p.nz + p.zchunk - 1) / p.zchunk;
      p.nunits = ntiles * nzc;
      *blocks = p.nunits;
    }
  }

  static cudaError_t run(const StepArgs& a, const Op& op, int* blocks_out) {
    TmaParams<Op, T> p;
    p.op = op;
    for (int f = 0; f < Op::NF; ++f) p.out[f] = static_cast<T*>(a.out[f]);
    p.partials = a.partials;
    p.err = a.err;
    int blocks = 0;
    geometry(a, p, &blocks);
    if (blocks_out) *blocks_out = blocks;
    if (Op::REDUCES && (!a.partials || blocks > a.partial_count)) return cudaErrorInvalidValue;
    TmaMaps<Op::NF> maps;
    const int64_t n[3] = {a.g.n[2], a.g.n[1], a.g.n[0]};
    for (int f = 0; f < Op::NF; ++f) {
      cudaError_t e;
      if ((e = encode<T>(&maps.main[f], a.in[f], RANK, n, TX, kTy + 2 * Op::R)) ||
          (e = encode<T>(&maps.body[f], a.in[f], RANK, n, TX, kTy)) ||
          (e = encode<T>(&maps.row[f], a.in[f], RANK, n, TX, 1)) ||
          (e = encode<T>(&maps.cols[f], a.in[f], RANK, n, L::CW, kTy)))
        return e;
    }
    occupancy();
    kernel()<<<blocks, THREADS, SMEM, a.stream>>>(maps, p);
    count_launches(1);
    return cudaGetLastError();
  }
};

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
  switch (s.kind) {
    case kJacobi5: return TmaRunner<OpJacobi5, T, 2>::run(a, {s.prm[0]}, blocks);
    case kStar9r2: return TmaRunner<OpStar9r2, T, 2>::run(a, {s.prm[0]}, blocks);
    case kDiff7: return TmaRunner<OpDiff7, T, 3>::run(a, {s.prm[0]}, blocks);
    case kSwe: return TmaRunner<OpSwe, T, 2>::run(a, {s.prm[0] * s.prm[2], s.prm[0] * s.prm[1]}, blocks);
    case kLinear: {
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
  if (!s.star || a.ksteps != 1 || s.radius < 1 || s.radius > 2) return false;
  if (s.kind == kSwe && g.ndim != 2) return false;
  const int esz = g.dtype == kF64 ? 8 : g.dtype == kF32 ? 4 : 2;
  const int cw = 16 / esz;
  if ((g.n[2] * esz) % 16 != 0) return false;
  for (int ax = 0; ax < 3; ++ax) {
    if (g.n[ax] > (int64_t(1) << 30)) return false;
    for (int sd = 0; sd < 2; ++sd) {
      if (g.bc[ax][sd] == kDirichlet && g.bval[ax][sd] != 0.0 && !a.adjoint) return false;
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
