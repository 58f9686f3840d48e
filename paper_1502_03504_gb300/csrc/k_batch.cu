// Batched form: many independent grids of uneven sizes advanced together by
// one persistent, cooperatively launched kernel.
//
// The work list holds every (grid, tile) pair of the batch.  Each pass runs k
// fused sweeps on every tile (trap.cuh), then all blocks meet at a grid-wide
// barrier before the next pass reads what this one wrote — the one-GPU form
// of "all threads finish the loop body, then the halo transfer synchronises"
// (Sec. 3.2).  The barrier wait is bounded: after kWaitLimitNs it records a
// timeout in the error flag and the kernel returns.  Loads in later passes go
// through L2 (ld.global.cg), so no block reads a stale L1 line of data another
// block wrote in the previous pass.
#include <algorithm>
#include <type_traits>

#include "trap.cuh"

namespace lope {

namespace {

constexpr int kBatchThreads = 256;

__device__ __forceinline__ bool grid_sync(unsigned int* bar, unsigned int target, int* err,
                                          volatile int* s_abort, unsigned long long wait_ns,
                                          bool arrive) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (arrive) atomicAdd(bar, 1u);
    const uint64_t t0 = global_ns();
    for (;;) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (global_ns() - t0 > wait_ns) {
        raise_error(err, kErrTimeout);
        *s_abort = 1;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return *s_abort == 0;
}

__device__ __forceinline__ int find_grid(const BatchGrid* grids, int ngrids, int item) {
  int lo = 0, hi = ngrids - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (grids[mid].first_item <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Tile policies: the variable-shape trapezoid (any tile and depth), or the
// shape fixed at compile time (TrapFixed: every tap at an immediate offset).
struct TileAny {
  template <class Op, class T>
  static __device__ __forceinline__ void run(const Op& op, const T* const* src, T* const* dst,
                                             const TrapGrid& g, int x0, int y0, int tx, int ty,
                                             int kp, C_t<T>* smem) {
    trap_tile<Op, T>(op, src, dst, g, x0, y0, tx, ty, kp, smem);
  }
};
template <int TX, int TY, int K>
struct TileFixed {
  template <class Op, class T>
  static __device__ __forceinline__ void run(const Op& op, const T* const* src, T* const* dst,
                                             const TrapGrid& g, int x0, int y0, int, int, int kp,
                                             C_t<T>* smem) {
    TrapFixed<Op, T, TX, TY, K>::tile(op, src, dst, g, x0, y0, kp, smem);
  }
};

template <class Op, class T, class Tile>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(Op op, BatchPlanDev p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ volatile int s_abort;
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();
  const int64_t passes = (p.nsteps + p.ksteps - 1) / p.ksteps;
  for (int64_t pass = 0; pass < passes; ++pass) {
    const int64_t rem = p.nsteps - pass * p.ksteps;
    const int kp = int(rem < p.ksteps ? rem : p.ksteps);
    const bool to_out = ((passes - 1 - pass) & 1) == 0;
    for (int item = blockIdx.x; item < p.nitems; item += gridDim.x) {
      const int gi = find_grid(p.grids, p.ngrids, item);
      const BatchGrid& bg = p.grids[gi];
      // pass 0 reads in; pass q > 0 reads what pass q-1 wrote
      const T* src = pass == 0 ? static_cast<const T*>(bg.in)
                               : static_cast<const T*>(to_out ? bg.work : bg.out);
      T* dst = static_cast<T*>(to_out ? bg.out : bg.work);
      const int t = item - bg.first_item;
      const int x0 = (t % bg.tiles_x) * p.tile_x, y0 = (t / bg.tiles_x) * p.tile_y;
      TrapGrid tg;
      tg.nx = bg.nx;
      tg.ny = bg.ny;
      for (int a = 0; a < 2; ++a)
        for (int sd = 0; sd < 2; ++sd) {
          tg.bc[a][sd] = bg.bc[a][sd];
          tg.bval[a][sd] = bg.bval[a][sd];
        }
      const T* srcs[1] = {src};
      T* dsts[1] = {dst};
      Tile::template run<Op, T>(op, srcs, dsts, tg, x0, y0, p.tile_x, p.tile_y, kp,
                                reinterpret_cast<C_t<T>*>(smem_raw));
    }
    const bool arrive = !(pass == 0 && int(blockIdx.x) == p.skip_block);
    if (pass + 1 < passes &&
        !grid_sync(p.barrier, unsigned(pass + 1) * gridDim.x, p.err, &s_abort, p.wait_ns, arrive))
      return;
  }
}

template <class Op, class T, class Tile> struct BatchRunner {
  static cudaError_t prepare(size_t smem) {
    return cudaFuncSetAttribute(&batch_kernel<Op, T, Tile>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(smem));
  }
  static int max_blocks(size_t smem) {
    if (prepare(smem) != cudaSuccess) return 0;
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, &batch_kernel<Op, T, Tile>, kBatchThreads,
                                                      smem) != cudaSuccess)
      return 0;
    return occ * sms;
  }
  static cudaError_t launch(const Op& op, const BatchPlanDev& p, int blocks, size_t smem,
                            cudaStream_t st) {
    cudaError_t e = prepare(smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, &batch_kernel<Op, T, Tile>, op, p);
    count_launches(1);
    return e;
  }
};

template <class T, class F> auto with_op(const StencilDesc& s, F&& f) {
  if (s.kind == kJacobi5) return f(OpJacobi5{s.prm[0]});
  OpStarLinear<2, 1> op;
  for (int ax = 0; ax < 3; ++ax)
    for (int d = 0; d < 3; ++d) op.w[ax][d] = s.star_w[ax][d];
  return f(op);
}

// Run F with the tile policy for (tile_x, tile_y, k): the fixed shapes the
// batch autotuner tries for FP32 storage, else the variable-shape tile.
template <class T, class F>
auto with_tile(int tx, int ty, int k, F&& f) {
  if constexpr (std::is_same<T, float>::value) {
#define LOPE_FIXED(X, Y, KK) \
    if (tx == X && ty == Y && k == KK) return f(TileFixed<X, Y, KK>());
    LOPE_FIXED(128, 32, 4) LOPE_FIXED(128, 32, 2) LOPE_FIXED(64, 32, 4) LOPE_FIXED(64, 32, 2)
    LOPE_FIXED(128, 16, 4) LOPE_FIXED(128, 16, 2) LOPE_FIXED(64, 16, 4) LOPE_FIXED(64, 16, 2)
#undef LOPE_FIXED
  }
  return f(TileAny());
}

template <class T>
cudaError_t launch_t(const BatchPlanDev& p, const StencilDesc& s, int blocks, cudaStream_t st) {
  const size_t smem = trap_smem_bytes(sizeof(T) == 8 ? kF64 : kF32, 1, p.tile_x, p.tile_y,
                                      s.radius * p.ksteps);
  return with_op<T>(s, [&](auto op) {
    return with_tile<T>(p.tile_x, p.tile_y, p.ksteps, [&](auto tile) {
      return BatchRunner<decltype(op), T, decltype(tile)>::launch(op, p, blocks, smem, st);
    });
  });
}

template <class T> int max_blocks_t(const StencilDesc& s, int tx, int ty, int k) {
  const size_t smem = trap_smem_bytes(sizeof(T) == 8 ? kF64 : kF32, 1, tx, ty, s.radius * k);
  return with_op<T>(s, [&](auto op) {
    return with_tile<T>(tx, ty, k, [&](auto tile) {
      return BatchRunner<decltype(op), T, decltype(tile)>::max_blocks(smem);
    });
  });
}

}  // namespace

cudaError_t launch_batch(const BatchPlanDev& p, const StencilDesc& s, int dtype, int blocks,
                         cudaStream_t st) {
  if (!(s.kind == kJacobi5 || (s.kind == kLinear && s.star && s.ndim == 2 && s.radius == 1)))
    return cudaErrorNotSupported;
  switch (dtype) {
    case kF32: return launch_t<float>(p, s, blocks, st);
    case kF64: return launch_t<double>(p, s, blocks, st);
    case kBF16: return launch_t<__nv_bfloat16>(p, s, blocks, st);
    default: return cudaErrorNotSupported;
  }
}

int batch_max_blocks(const StencilDesc& s, int dtype, int tile_x, int tile_y, int ksteps) {
  if (!(s.kind == kJacobi5 || (s.kind == kLinear && s.star && s.ndim == 2 && s.radius == 1)))
    return 0;
  switch (dtype) {
    case kF32: return max_blocks_t<float>(s, tile_x, tile_y, ksteps);
    case kF64: return max_blocks_t<double>(s, tile_x, tile_y, ksteps);
    case kBF16: return max_blocks_t<__nv_bfloat16>(s, tile_x, tile_y, ksteps);
    default: return 0;
  }
}

}  // namespace lope
