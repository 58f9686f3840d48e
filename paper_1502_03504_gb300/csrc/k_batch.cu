// Batched form: many independent grids of uneven sizes advanced together by
// one persistent, cooperatively launched kernel.
//
// The work list holds every (grid, tile) pair of the batch.  Each pass runs k
// fused sweeps on every tile (trap.cuh), then all blocks meet at a grid-wide
// barrier before the next pass reads what this one wrote — the one-GPU form
// of "all threads finish the loop body, then the halo transfer synchronises"
// (Sec. 3.2).  The barrier wait is bounded: after kWaitLimitNs it records a
// timeout in the error flag and the kernel returns.  The barrier's GPU-scope
// acquire, passed on to the whole block by its CTA barrier, orders every read
// of the next pass (the asynchronous window copies included) after the stores
// every block made in this one.
#include <algorithm>
#include <type_traits>

#include "tma_device.cuh"
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

// ------------------------------------------------------------------ two sweeps per pass
// The batched form of the two-sweep 2D tiles (tma2d_tb2_kernel), for FP32 grids
// of any row pitch: a 64 x TY tile is staged into shared memory with a 2R-row
// / 4-column halo by 4-byte asynchronous copies (cp.async; the grids' rows need
// not be 16-byte aligned, as TMA would require), the boundary rule applied as
// each cell is staged (rows first: the Dirichlet value, stored directly, or
// the wrapped row; then columns likewise); the first sweep u1 is computed on
// the tile and its R-wide ring and held at the side's Dirichlet value past a
// Dirichlet side; the second sweep writes the tile.
//
// Two staging boxes alternate: the copies of the next tile are issued before
// the first sweep of the current one, so they have a whole tile's sweeps to
// land.  Tiles are claimed one at a time from a counter, two ahead of the
// tile being swept, and each claimed tile's 64-byte record (BatchItem) is
// read while the current tile's second sweep runs.  A pass (two sweeps, or
// one for the last of an odd count) covers every tile of every grid; passes
// are separated by the bounded grid-wide barrier, whose acquire orders the
// next pass's copies after every block's stores.  All threads of a block run
// the same control flow, so its barriers cannot strand a thread.
template <int R>
struct BatchTb2Geom {
  static constexpr int TX = 64, H = 2 * R, CW = 4, W = TX + 2 * CW;  // box columns -4..TX+3
  static constexpr int W1 = TX + 4;                                   // u1 columns -2..TX+1
  static constexpr __host__ __device__ int box_floats(int ty) { return (ty + 2 * H) * W; }
  static constexpr __host__ __device__ int u1_floats(int ty) { return (ty + 2 * R) * W1; }
};

// Fill the tile records of the two-sweep batched tiles from the grid list.
__global__ void batch_items_kernel(const BatchGrid* grids, int ngrids, int nitems, int tx, int ty,
                                   BatchItem* items) {
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < nitems; it += gridDim.x * blockDim.x) {
    const BatchGrid& g = grids[find_grid(grids, ngrids, it)];
    const int t = it - g.first_item;
    BatchItem b;
    b.in = static_cast<const float*>(g.in);
    b.out = static_cast<float*>(g.out);
    b.work = static_cast<float*>(g.work);
    b.nx = g.nx;
    b.ny = g.ny;
    b.x0 = (t % g.tiles_x) * tx;
    b.y0 = (t / g.tiles_x) * ty;
    b.bc = (g.bc[0][0] & 255) | (g.bc[0][1] & 255) << 8 | (g.bc[1][0] & 255) << 16 |
           (g.bc[1][1] & 255) << 24;
    b.vy0 = float(g.bval[0][0]);
    b.vy1 = float(g.bval[0][1]);
    b.vx0 = float(g.bval[1][0]);
    b.vx1 = float(g.bval[1][1]);
    b.pad = 0;
    items[it] = b;
  }
}

template <class Op, int TY, int RY>
__global__ void __launch_bounds__(32 * (TY / RY), 3) batch_tb2_kernel(Op op, BatchPlanDev p) {
  using G = BatchTb2Geom<Op::R>;
  constexpr int TX = G::TX, R = Op::R, H = G::H, CW = G::CW, W = G::W, W1 = G::W1;
  static_assert(Op::NF == 1 && Op::STAR && R <= 2, "radius <= 2 star function of one field");
  constexpr int BH = TY + 2 * H, NW = TY / RY, NT = 32 * NW;
  constexpr int NC = RY + 2 * R, BOXN = G::box_floats(TY);
  constexpr int NRING = 2 * R * 32 + 2 * TY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* const boxes = reinterpret_cast<float*>(smem_raw);  // two staging boxes
  float* const u1 = boxes + 2 * BOXN;
  // Tile records: the tile being swept, the next one (staged during this
  // tile's sweeps) and the one after (fetched during the second sweep).
  __shared__ __align__(16) BatchItem s_rec[3];
  __shared__ volatile int s_abort;
  __shared__ int s_claim;
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  const int cx2 = lane * 2, cy0 = warp * RY;
  if (tid == 0) s_abort = 0;
  __syncthreads();
  // Threads 0-3 copy the four 16-byte quarters of a record into slot `sl`
  // (asynchronously; the copy lands by the next wait).
  auto fetch_rec = [&](int item, int sl) {
    if (item >= 0 && tid < 4) {
      const uint32_t d = smem_u32(&s_rec[sl]) + 16u * unsigned(tid);
      const char* src = reinterpret_cast<const char*>(p.items + item) + 16 * tid;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  const int64_t passes = (p.nsteps + 1) / 2;
  for (int64_t pass = 0; pass < passes; ++pass) {
    const int kp = (pass == passes - 1 && (p.nsteps & 1)) ? 1 : 2;
    const bool to_out = ((passes - 1 - pass) & 1) == 0;
    // Each block claims until its first claim past the list and then once
    // more (the claims run two tiles ahead), so each pass takes exactly
    // nitems + 2 * gridDim.x claims and pass `pass` starts from
    // pass * (nitems + 2 * gridDim.x).
    const unsigned long long pbase =
        (unsigned long long)pass * (unsigned long long)(p.nitems + 2 * int(gridDim.x));
    auto claim_raw = [&]() { return atomicAdd(p.claim, 1ull) - pbase; };
    auto valid = [&](unsigned long long v) { return v < (unsigned long long)p.nitems ? int(v) : -1; };
    // Stage the tile of record `t` into `box`: warp w takes box rows w,
    // w + NW, ...; lane l the box columns l, l + 32, l + 64.  A tile whose box
    // lies inside its grid copies every cell; elsewhere the row rule is
    // decided once per row and the column rule once per column, rows (the
    // slower axis) first.  Ends with a commit, so each tile's copies form
    // one group.
    auto load = [&](const BatchItem& t, float* box) {
      const uint32_t sbox = smem_u32(box);
      const float* src = pass == 0 ? t.in : (to_out ? t.work : t.out);
      const int nx = t.nx, ny = t.ny, x0 = t.x0, y0 = t.y0;
      if (x0 >= CW && x0 + TX + CW <= nx && y0 >= H && y0 + TY + H <= ny) {
        // a box row is a run of consecutive cells: 16- or 8-byte copies where
        // the run's first cell is so aligned (box rows are 16-byte aligned)
        const float* r0 = src + int64_t(y0 - H + warp) * nx + (x0 - CW);
        const int64_t step = int64_t(NW) * nx;
        uint32_t d = sbox + 4u * unsigned(warp * W);
        static_assert(W % 4 == 0 && W / 4 <= 32 && W / 2 <= 64 && W <= 96, "box row copies");
#pragma unroll 4
        for (int br = warp; br < BH; br += NW, r0 += step, d += 4u * NW * W) {
          const unsigned mis = unsigned(reinterpret_cast<uintptr_t>(r0)) & 15u;
          if (mis == 0) {
            if (lane < W / 4) cp_async_16(d + 16u * lane, r0 + 4 * lane);
          } else if ((mis & 7u) == 0) {
            cp_async_elem<8>(d + 8u * lane, r0 + 2 * lane);
            if (lane < W / 2 - 32) cp_async_elem<8>(d + 8u * (lane + 32), r0 + 2 * (lane + 32));
          } else {
            cp_async_elem<4>(d + 4u * lane, r0 + lane);
            cp_async_elem<4>(d + 4u * (lane + 32), r0 + lane + 32);
            if (lane < W - 64) cp_async_elem<4>(d + 4u * (lane + 64), r0 + lane + 64);
          }
        }
      } else {
        const int bcy0 = t.bc & 255, bcy1 = (t.bc >> 8) & 255;
        const int bcx0 = (t.bc >> 16) & 255, bcx1 = (t.bc >> 24) & 255;
        int gcol[3];
        float cval[3];
        bool cfix[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          int gx = x0 - CW + lane + 32 * k;
          cfix[k] = false;
          cval[k] = 0.f;
          if (gx < 0 || gx >= nx) {
            const bool lo = gx < 0;
            if ((lo ? bcx0 : bcx1) == kDirichlet) {
              cfix[k] = true;
              cval[k] = lo ? t.vx0 : t.vx1;
            }
            gx = wrap(gx, nx);
          }
          gcol[k] = gx;
        }
        for (int br = warp; br < BH; br += NW) {
          int gy = y0 - H + br;
          bool rfix = false;
          float rval = 0.f;
          if (gy < 0 || gy >= ny) {
            const bool lo = gy < 0;
            if ((lo ? bcy0 : bcy1) == kDirichlet) {
              rfix = true;
              rval = lo ? t.vy0 : t.vy1;
            }
            gy = wrap(gy, ny);
          }
          const float* row = src + int64_t(gy) * nx;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            if (lane + 32 * k >= W) break;
            const int at = br * W + lane + 32 * k;
            if (rfix) box[at] = rval;
            else if (cfix[k]) box[at] = cval[k];
            else cp_async_elem<4>(sbox + 4u * unsigned(at), row + gcol[k]);
          }
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // Prologue: the first tile claimed, its record read and its box staged;
    // the second claimed and its record fetched.
    if (tid == 0) s_claim = valid(claim_raw());
    __syncthreads();
    int cur = s_claim;
    fetch_rec(cur, 0);
    cp_async_wait_all();
    __syncthreads();  // the record is visible; every thread has read s_claim
    if (tid == 0) s_claim = valid(claim_raw());
    if (cur >= 0) load(s_rec[0], boxes);
    __syncthreads();
    int nxt = s_claim;
    fetch_rec(nxt, 1);
    int a = 0, b = 1, c = 2, buf = 0;
    while (cur >= 0) {
      cp_async_wait_all();
      __syncthreads();  // this tile's box and the next record have landed; u1 is free
      // the next tile's copies go to the other box, free since the barrier
      // after the previous tile's first sweep
      if (nxt >= 0) load(s_rec[b], boxes + (buf ^ 1) * BOXN);
      unsigned long long v = 0;
      if (tid == 0) v = claim_raw();  // the tile after next; published after the first sweep
      const BatchItem& t = s_rec[a];
      const float* box = boxes + buf * BOXN;
      const int nx = t.nx, ny = t.ny, x0 = t.x0, y0 = t.y0;
      const bool edge = x0 < CW || x0 + TX + CW > nx || y0 < H || y0 + TY + H > ny;
      auto sweep1 = [&](auto edge_tag) {
        constexpr bool EDGE = decltype(edge_tag)::value;
        // Cells past a Dirichlet side keep its value: tile rows outside
        // [row_lo, row_hi) and columns outside [col_lo, col_hi) (rows first,
        // then columns, the order of the boundary rule).
        constexpr int kFar = 1 << 30;
        int row_lo = -kFar, row_hi = kFar, col_lo = -kFar, col_hi = kFar;
        float vy0 = 0.f, vy1 = 0.f, vx0 = 0.f, vx1 = 0.f;
        if constexpr (EDGE) {
          if ((t.bc & 255) == kDirichlet) row_lo = -y0;
          if (((t.bc >> 8) & 255) == kDirichlet) row_hi = ny - y0;
          if (((t.bc >> 16) & 255) == kDirichlet) col_lo = -x0;
          if (((t.bc >> 24) & 255) == kDirichlet) col_hi = nx - x0;
          vy0 = t.vy0;
          vy1 = t.vy1;
          vx0 = t.vx0;
          vx1 = t.vx1;
        }
        auto cell = [&](float v, int tc) { return tc < col_lo ? vx0 : tc >= col_hi ? vx1 : v; };
        auto mask = [&](F2 v, int tr, int tc) {
          if (tr < row_lo) return F2::make(vy0, vy0);
          if (tr >= row_hi) return F2::make(vy1, vy1);
          return F2::make(cell(v.lo(), tc), cell(v.hi(), tc + 1));
        };
        F2 col[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) col[k] = ld_pair(box + (H - R + cy0 + k) * W + CW + cx2);
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          PairAcc<float, TX, TY, R, 1, NC> acc;
          acc.b[0] = box + (H + cy0 + r) * W + CW + cx2;
          acc.col = &col;
          acc.r = r;
          acc.g = 0;
          F2 o[1];
          F2 unused(0.f);
          op(acc, o, unused);
          F2 v = o[0];
          if constexpr (EDGE) v = mask(v, cy0 + r, cx2);
          st_pair_f(u1 + (R + cy0 + r) * W1 + 2 + cx2, v);
        }
        for (int q = tid; q < NRING; q += NT) {
          int tr, tc;
          if (q < 2 * R * 32) {
            const int row = q >> 5;
            tr = row < R ? row - R : TY + row - R;
            tc = (q & 31) * 2;
          } else {
            const int d = q - 2 * R * 32;
            tr = d >> 1;
            tc = (d & 1) ? TX : -2;
          }
          Smem2Acc<float, W> acc{box + (H + tr) * W + CW + tc};
          F2 o[1];
          F2 unused(0.f);
          op(acc, o, unused);
          F2 v = o[0];
          if constexpr (EDGE) v = mask(v, tr, tc);
          st_pair_f(u1 + (R + tr) * W1 + 2 + tc, v);
        }
      };
      if (edge) sweep1(BoolTag<true>());
      else sweep1(BoolTag<false>());
      if (tid == 0) s_claim = valid(v);
      __syncthreads();  // u1 complete; s_claim published; this box is free
      const int nn = s_claim;
      fetch_rec(nn, c);  // the record slot of the previous tile, read before the barrier above
      float* const out = to_out ? t.out : t.work;
      const int ox = x0 + cx2, oy = y0 + cy0;
      auto put = [&](int r, F2 v) {
        const int gy = oy + r;
        if (gy >= ny || ox >= nx) return;
        float* d = out + int64_t(gy) * nx + ox;
        if (ox + 1 < nx && (reinterpret_cast<uintptr_t>(d) & 7) == 0) {
          st_pair(d, v);
        } else {
          d[0] = v.lo();
          if (ox + 1 < nx) d[1] = v.hi();
        }
      };
      if (kp == 1) {  // a one-sweep pass: u1 is the result
#pragma unroll
        for (int r = 0; r < RY; ++r) put(r, ld_pair(u1 + (R + cy0 + r) * W1 + 2 + cx2));
      } else {
        F2 col[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) col[k] = ld_pair(u1 + (cy0 + k) * W1 + 2 + cx2);
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          PairAcc<float, TX, TY, R, 1, NC> acc;
          acc.b[0] = u1 + (R + cy0 + r) * W1 + 2 + cx2;
          acc.col = &col;
          acc.r = r;
          acc.g = 0;
          F2 o[1];
          F2 unused(0.f);
          op(acc, o, unused);
          put(r, o[0]);
        }
      }
      cur = nxt;
      nxt = nn;
      const int a0 = a;
      a = b;
      b = c;
      c = a0;
      buf ^= 1;
    }
    cp_async_wait_all();
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

// Two-sweep register tiles: 8 warps of 8 rows on 64 x 64 tiles, three blocks
// per SM, each with two staging boxes (measured on the 512-grid workload:
// 12.3 ms for 20 sweeps against 15.0 ms on 64 x 128 tiles with two blocks of
// 8 warps of 16 rows, and 14.4 ms with two blocks of 16 warps of 8 rows).
constexpr int kTb2RY = 8, kTb2Threads = 32 * (kBatchTb2Y / kTb2RY);

template <class Op>
size_t tb2_smem() {
  using G = BatchTb2Geom<Op::R>;
  return size_t(2 * G::box_floats(kBatchTb2Y) + G::u1_floats(kBatchTb2Y)) * 4;
}

template <class Op>
struct BatchTb2Runner {
  static auto kernel() { return &batch_tb2_kernel<Op, kBatchTb2Y, kTb2RY>; }
  static int max_blocks() {
    if (cudaFuncSetAttribute(kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(tb2_smem<Op>())) != cudaSuccess)
      return 0;
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel(), kTb2Threads, tb2_smem<Op>()) !=
        cudaSuccess)
      return 0;
    return occ * sms;
  }
  static cudaError_t launch(const Op& op, const BatchPlanDev& p, int blocks, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(tb2_smem<Op>()));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kTb2Threads);
    cfg.dynamicSmemBytes = tb2_smem<Op>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the tile records first (one thread per tile), then the persistent kernel
    batch_items_kernel<<<(p.nitems + 255) / 256, 256, 0, st>>>(p.grids, p.ngrids, p.nitems,
                                                               kBatchTb2X, kBatchTb2Y, p.items);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernelEx(&cfg, kernel(), op, p);
    count_launches(2);
    return e;
  }
};

// Local functions of the two-sweep batched tiles: the 5-point Jacobi, the
// 9-point radius-2 star, and linear star tables of radius 1 or 2.
template <class F> cudaError_t with_tb2_op(const StencilDesc& s, F&& f) {
  if (s.kind == kJacobi5) return f(OpJacobi5{s.prm[0]});
  if (s.kind == kStar9r2) return f(OpStar9r2{s.prm[0]});
  if (s.kind == kLinear && s.star && s.ndim == 2 && s.radius == 1) {
    OpStarLinear<2, 1> op;
    for (int ax = 0; ax < 3; ++ax) for (int d = 0; d < 3; ++d) op.w[ax][d] = s.star_w[ax][d];
    return f(op);
  }
  if (s.kind == kLinear && s.star && s.ndim == 2 && s.radius == 2) {
    OpStarLinear<2, 2> op;
    for (int ax = 0; ax < 3; ++ax) for (int d = 0; d < 5; ++d) op.w[ax][d] = s.star_w[ax][d];
    return f(op);
  }
  return cudaErrorNotSupported;
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
  if (p.mode == 1) {
    if (dtype != kF32) return cudaErrorNotSupported;
    return with_tb2_op(s, [&](auto op) {
      return BatchTb2Runner<decltype(op)>::launch(op, p, blocks, st);
    });
  }
  if (!(s.kind == kJacobi5 || (s.kind == kLinear && s.star && s.ndim == 2 && s.radius == 1)))
    return cudaErrorNotSupported;
  switch (dtype) {
    case kF32: return launch_t<float>(p, s, blocks, st);
    case kF64: return launch_t<double>(p, s, blocks, st);
    case kBF16: return launch_t<__nv_bfloat16>(p, s, blocks, st);
    default: return cudaErrorNotSupported;
  }
}

int batch_max_blocks(const StencilDesc& s, int dtype, int tile_x, int tile_y, int ksteps,
                     int mode) {
  if (mode == 1) {
    if (dtype != kF32 || tile_x != kBatchTb2X || tile_y != kBatchTb2Y || ksteps < 1 || ksteps > 2)
      return 0;
    int b = 0;
    with_tb2_op(s, [&](auto op) {
      b = BatchTb2Runner<decltype(op)>::max_blocks();
      return cudaSuccess;
    });
    return b;
  }
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
