// Device-side building blocks shared by the LOPe kernels: storage/compute
// types, explicitly rounded arithmetic, mbarrier and TMA wrappers (inline PTX
// for sm_103a), bounded waits, and the local functions themselves.
#pragma once

#ifdef __CUDACC_RTC__
// Run-time compilation (NVRTC): the fixed-width integer types and the opaque
// 128-byte tensor-map type the kernels take by value, declared as the CUDA
// headers declare them.
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long int64_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long uint64_t;
typedef unsigned long uintptr_t;
typedef struct alignas(64) CUtensorMap_st { unsigned long long opaque[16]; } CUtensorMap;
#include <cuda_bf16.h>
#else
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "lope_internal.h"

namespace lope {

// ---------------------------------------------------------------- types
template <class T> struct Compute { using type = float; };
template <> struct Compute<double> { using type = double; };
template <class T> using C_t = typename Compute<T>::type;

__device__ __forceinline__ double to_c(double v) { return v; }
__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class T> __device__ __forceinline__ T from_c(C_t<T> v);
template <> __device__ __forceinline__ double from_c<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_c<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_c<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
// Round a compute value to what storage would hold (identity for f32/f64).
template <class T> __device__ __forceinline__ C_t<T> to_storage_precision(C_t<T> v) {
  return to_c(from_c<T>(v));
}

// Explicitly rounded arithmetic: every kernel variant evaluates a local
// function with the same operations in the same order, so results are
// bitwise identical across tilings and temporal depths.
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

// Two FP32 values in one 64-bit register, operated on by the packed f32x2
// instructions of sm_100-family GPUs (each lane is an IEEE round-to-nearest
// operation, so a pair gives bitwise the results of two scalar operations).
// Local functions written against add/sub/mul/fma_ and C(constant) run
// unchanged on pairs: a kernel then computes two adjacent columns at once.
struct F2 {
  uint64_t v;
  F2() = default;
  __device__ __forceinline__ explicit F2(float a) {
    asm("mov.b64 %0, {%1, %1};" : "=l"(v) : "f"(a));
  }
  __device__ __forceinline__ static F2 make(float lo, float hi) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
  }
  __device__ __forceinline__ float lo() const {
    float a;
    asm("{\n\t.reg .b32 t;\n\tmov.b64 {%0, t}, %1;\n\t}" : "=f"(a) : "l"(v));
    return a;
  }
  __device__ __forceinline__ float hi() const {
    float b;
    asm("{\n\t.reg .b32 t;\n\tmov.b64 {t, %0}, %1;\n\t}" : "=f"(b) : "l"(v));
    return b;
  }
};

__device__ __forceinline__ F2 add(F2 a, F2 b) {
  F2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ F2 sub(F2 a, F2 b) {
  F2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
// The packed product is an FMA with a -0 addend (a*b + -0 = a*b exactly, with
// the sign of a zero product kept).  ptxas contracts a packed mul.rn followed
// by a packed add/sub into a single FMA despite the rounding qualifier, and
// it can still do so with this form (measured on sm_103a: sub(s, mul(3, u))
// gave fma(-3, u, s) at every point where the two differ), so a product that
// feeds a sum may round once less than on the scalar paths.  The builtins
// write such products as fma_, which rounds alike on every path.
__device__ __forceinline__ F2 mul(F2 a, F2 b) {
  F2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(0x8000000080000000ull));
  return d;
}
__device__ __forceinline__ F2 fma_(F2 a, F2 b, F2 c) {
  F2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}

// Operators on packed pairs, for local functions written with + - * (user
// source compiled at run time); they are the explicitly rounded operations
// above.  Negation flips the sign bits (exact).
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return add(a, b); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return sub(a, b); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return mul(a, b); }
__device__ __forceinline__ F2 operator-(F2 a) {
  F2 d;
  asm("xor.b64 %0, %1, 0x8000000080000000;" : "=l"(d.v) : "l"(a.v));
  return d;
}

// Load a stored value (or an aligned pair of adjacent values) of global memory
// in compute precision.
__device__ __forceinline__ float ldc(const float* p, float) { return __ldg(p); }
__device__ __forceinline__ float ldc(const __nv_bfloat16* p, float) { return __bfloat162float(p[0]); }
__device__ __forceinline__ double ldc(const double* p, double) { return __ldg(p); }
__device__ __forceinline__ F2 ldc(const float* p, F2) {
  F2 r;
  r.v = __ldg(reinterpret_cast<const unsigned long long*>(p));
  return r;
}
__device__ __forceinline__ F2 ldc(const __nv_bfloat16* p, F2) {
  const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  return F2::make(f.x, f.y);
}

// ---------------------------------------------------------------- timers / waits
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Record a timeout in the device error flag (first writer wins).
__device__ __forceinline__ void raise_error(int* flag, int code) {
  if (flag) atomicCAS(flag, 0, code);
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Asynchronous copy of one 4- or 8-byte element from global to shared memory
// (cp.async through L1 and L2, 128-byte L2 fetches).  Many can be in flight
// per thread; they complete at cp_async_wait_all.
template <int B>
__device__ __forceinline__ void cp_async_elem(uint32_t dst, const void* src) {
  static_assert(B == 4 || B == 8, "element copies of 4 or 8 bytes");
  if constexpr (B == 4)
    asm volatile("cp.async.ca.shared.global.L2::128B [%0], [%1], 4;" ::"r"(dst), "l"(src)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global.L2::128B [%0], [%1], 8;" ::"r"(dst), "l"(src)
                 : "memory");
}
// One 16-byte asynchronous copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async_16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global.L2::128B [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// One try_wait with a suspend-time hint: the thread may sleep in hardware
// until the phase completes or about kSuspendNs pass, instead of spinning and
// taking issue slots from the warps that have work.
constexpr uint32_t kSuspendNs = 20000;

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}

// Non-blocking probe of a phase.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the given phase parity with a time limit.  Returns false (and the
// caller must stop) when the limit passes; nothing here traps.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 15u) == 15u && global_ns() - t0 > kWaitLimitNs) {
      raise_error(err, kErrTimeout);
      return false;
    }
  }
}

// ---------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* m) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* m, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* m, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ int wrap(int q, int n) {
  q %= n;
  return q < 0 ? q + n : q;
}

// Index of coordinate v (within one extent of the axis, -n <= v < 2n) on an
// axis of extent n: itself when inside, wrapped on a periodic side, or -1 / -2
// past a low / high Dirichlet side.
__device__ __forceinline__ int axis_index(int v, int n, int bc_lo, int bc_hi) {
  if (v < 0) return bc_lo == kDirichlet ? -1 : v + n;
  if (v >= n) return bc_hi == kDirichlet ? -2 : v - n;
  return v;
}

// A coefficient kept in both precisions, converted once on the host (round
// to nearest), so FP32 kernels never convert FP64 values per point.
struct Coef {
  double d;
  float f;
  Coef() = default;
  __host__ __device__ Coef(double v) : d(v), f(float(v)) {}
  __device__ __forceinline__ float get(float) const { return f; }
  __device__ __forceinline__ double get(double) const { return d; }
  __device__ __forceinline__ F2 get(F2) const { return F2(f); }
};

// ---------------------------------------------------------------- local functions
//
// Each local function writes only its own element(s) and reads U(f,dx,dy,dz)
// through an accessor that hides where the halo values come from (shared
// memory tile, register queue, global memory with boundary logic).  This is
// the LOPe contract (Sec. 2.2, Fig. 1): the function never sees where its
// element sits in the grid.  The `red` argument (compute precision) receives
// a per-point term that only the adjoint functions produce; the kernels sum
// those terms over a few points and then accumulate in FP64.

struct OpJacobi5 {  // Fig. 1 with a coefficient: u + c (E + W + N + S - 4u)
  static constexpr int NDIM = 2, R = 1, NF = 1;
  static constexpr bool REDUCES = false, STAR = true;
  Coef c;
  template <class C, class A>
  __device__ __forceinline__ void operator()(const A& U, C (&o)[1], C&) const {
    C u = U(0, 0, 0, 0);
    C nb = add(add(U(0, -1, 0, 0), U(0, 1, 0, 0)), add(U(0, 0, -1, 0), U(0, 0, 1, 0)));
    o[0] = fma_(c.get(C()), fma_(C(-4), u, nb), u);
  }
};

struct OpDiff7 {  // u + c (sum of the six face neighbours - 6u)
  static constexpr int NDIM = 3, R = 1, NF = 1;
  static constexpr bool REDUCES = false, STAR = true;
  Coef c;
  template <class C, class A>
  __device__ __forceinline__ void operator()(const A& U, C (&o)[1], C&) const {
    C u = U(0, 0, 0, 0);
    C nb = add(add(add(U(0, -1, 0, 0), U(0, 1, 0, 0)), add(U(0, 0, -1, 0), U(0, 0, 1, 0))),
               add(U(0, 0, 0, -1), U(0, 0, 0, 1)));
    o[0] = fma_(c.get(C()), fma_(C(-6), u, nb), u);
  }
};

struct OpStar9r2 {  // u + c (L4x u + L4y u), L4 = (-1/12, 4/3, -5/2, 4/3, -1/12)
  static constexpr int NDIM = 2, R = 2, NF = 1;
  static constexpr bool REDUCES = false, STAR = true;
  Coef c;
  template <class C, class A>
  __device__ __forceinline__ void operator()(const A& U, C (&o)[1], C&) const {
    C u = U(0, 0, 0, 0);
    C s1 = add(add(U(0, -1, 0, 0), U(0, 1, 0, 0)), add(U(0, 0, -1, 0), U(0, 0, 1, 0)));
    C s2 = add(add(U(0, -2, 0, 0), U(0, 2, 0, 0)), add(U(0, 0, -2, 0), U(0, 0, 2, 0)));
    C lap = fma_(C(4.0 / 3.0), s1, fma_(C(-1.0 / 12.0), s2, mul(C(-5), u)));
    o[0] = fma_(c.get(C()), lap, u);
  }
};

// Linearised shallow water on an Arakawa C-grid (fields h, u, v): h at cell
// centres, u on east faces, v on north faces; forward Euler.
struct OpSwe {
  static constexpr int NDIM = 2, R = 1, NF = 3;
  static constexpr bool REDUCES = false, STAR = true;
  Coef mdtH, mdtg;  // -dt*H and -dt*g
  template <class C, class A>
  __device__ __forceinline__ void operator()(const A& U, C (&o)[3], C&) const {
    C h = U(0, 0, 0, 0), u = U(1, 0, 0, 0), v = U(2, 0, 0, 0);
    C div = add(sub(u, U(1, -1, 0, 0)), sub(v, U(2, 0, -1, 0)));
    o[0] = fma_(mdtH.get(C()), div, h);
    o[1] = fma_(mdtg.get(C()), sub(U(0, 1, 0, 0), h), u);
    o[2] = fma_(mdtg.get(C()), sub(U(0, 0, 1, 0), h), v);
  }
};

// Nonlinear shallow water on an Arakawa C-grid in flux form (fields eta =
// h - H, u, v; unit spacing; forward Euler).  Mass: eta' = eta - dt [F(i) -
// F(i-1) + G(j) - G(j-1)] with F = (H + face mean of eta) u and G likewise
// with v.  Momentum: Coriolis on the four-face means vbar / ubar (which read
// the corner taps U(+1,-1) of v and U(-1,+1) of u), the pressure gradient,
// and centred advection u D_x u + vbar D_y u (resp. ubar D_x v + v D_y v).
// A non-linear physics operator (Sec. 5, Limitations) written as one local
// function: products of halo values, three fields, a box halo.
//
// Every product that feeds a sum is written as an FMA (the flux differences
// below): the compiler may contract a packed multiply followed by a packed
// add into one FMA on its own, so leaving no such pair keeps the packed and
// scalar paths bitwise identical.
struct OpSweFlux {
  static constexpr int NDIM = 2, R = 1, NF = 3;
  static constexpr bool REDUCES = false, STAR = false;
  Coef dt, mdt, mg, f, mf, H, mH;  // dt, -dt, -g, f, -f, H, -H
  template <class C, class A>
  __device__ __forceinline__ void operator()(const A& U, C (&o)[3], C&) const {
    const C half = C(0.5f), quarter = C(0.25f), mhalf = C(-0.5f);
    const C h = H.get(C()), mh = mH.get(C());
    const C e = U(0, 0, 0, 0), eE = U(0, 1, 0, 0), eW = U(0, -1, 0, 0);
    const C eN = U(0, 0, 1, 0), eS = U(0, 0, -1, 0);
    const C u = U(1, 0, 0, 0), uW = U(1, -1, 0, 0), uE = U(1, 1, 0, 0);
    const C uN = U(1, 0, 1, 0), uS = U(1, 0, -1, 0), uWN = U(1, -1, 1, 0);
    const C v = U(2, 0, 0, 0), vS = U(2, 0, -1, 0), vN = U(2, 0, 1, 0);
    const C vE = U(2, 1, 0, 0), vW = U(2, -1, 0, 0), vES = U(2, 1, -1, 0);
    // F(i) - F(i-1) = hbar_E u + (-hbar_W) u_W; the negated face depth is
    // computed with negated coefficients, which is exact.
    const C dF = fma_(fma_(half, add(e, eE), h), u, mul(fma_(mhalf, add(eW, e), mh), uW));
    const C dG = fma_(fma_(half, add(e, eN), h), v, mul(fma_(mhalf, add(eS, e), mh), vS));
    o[0] = fma_(mdt.get(C()), add(dF, dG), e);
    const C vbar = mul(quarter, add(add(v, vE), add(vS, vES)));
    const C ubar = mul(quarter, add(add(u, uW), add(uN, uWN)));
    const C au = mul(mhalf, fma_(u, sub(uE, uW), mul(vbar, sub(uN, uS))));
    const C tu = fma_(f.get(C()), vbar, fma_(mg.get(C()), sub(eE, e), au));
    o[1] = fma_(dt.get(C()), tu, u);
    const C av = mul(mhalf, fma_(ubar, sub(vE, vW), mul(v, sub(vN, vS))));
    const C tv = fma_(mf.get(C()), ubar, fma_(mg.get(C()), sub(eN, e), av));
    o[2] = fma_(dt.get(C()), tv, v);
  }
  static OpSweFlux make(const double* prm) {
    OpSweFlux op;
    op.dt = prm[0];
    op.mdt = -prm[0];
    op.mg = -prm[1];
    op.f = prm[2];
    op.mf = -prm[2];
    op.H = prm[3];
    op.mH = -prm[3];
    return op;
  }
};

// General linear star stencil: w[axis][d + R], axis 0 = x (fastest), 1 = y,
// 2 = z; the centre weight sits in w[0][R] only.
template <int ND, int RR>
struct OpStarLinear {
  static constexpr int NDIM = ND, R = RR, NF = 1;
  static constexpr bool REDUCES = false, STAR = true;
  Coef w[3][2 * RR + 1];
  template <class C, class A>
  __device__ __forceinline__ void operator()(const A& U, C (&o)[1], C&) const {
    C s = mul(w[0][RR].get(C()), U(0, 0, 0, 0));
#pragma unroll
    for (int d = -RR; d <= RR; ++d) {
      if (d == 0) continue;
      s = fma_(w[0][d + RR].get(C()), U(0, d, 0, 0), s);
      s = fma_(w[1][d + RR].get(C()), U(0, 0, d, 0), s);
      if (ND == 3) s = fma_(w[2][d + RR].get(C()), U(0, 0, 0, d), s);
    }
    o[0] = s;
  }
};

// General linear box stencil (corners allowed), weights slowest offset first.
template <int ND, int RR>
struct OpBoxLinear {
  static constexpr int NDIM = ND, R = RR, NF = 1;
  static constexpr bool REDUCES = false, STAR = false;
  static constexpr int SIDE = 2 * RR + 1;
  static constexpr int ZS = ND == 3 ? SIDE : 1;
  Coef w[ZS * SIDE * SIDE];
  template <class C, class A>
  __device__ __forceinline__ void operator()(const A& U, C (&o)[1], C&) const {
    C s = C(0);
    constexpr int ZR = ND == 3 ? RR : 0;
#pragma unroll
    for (int dz = -ZR; dz <= ZR; ++dz)
#pragma unroll
      for (int dy = -RR; dy <= RR; ++dy)
#pragma unroll
        for (int dx = -RR; dx <= RR; ++dx)
          s = fma_(w[((dz + ZR) * SIDE + dy + RR) * SIDE + dx + RR].get(C()), U(0, dx, dy, dz), s);
    o[0] = s;
  }
};

// Adjoint step of a diffusion-form stencil u' = u + c L u, run on lambda:
// lambda_t = lambda_{t+1} + c L^T lambda_{t+1}, with L^T the offset-reflected
// stencil (the offset sets of these stencils are symmetric, so the reflection
// maps each tap onto a tap of the same weight).  Accumulates
// <L^T lambda_{t+1}, u_t> = <lambda_{t+1}, L u_t> for dL/dc; u_t is read at
// the local element only.  Halo of lambda: zero on Dirichlet sides (A^T has no
// constant term), wrapped on periodic ones.
template <int KIND, class T>
struct OpAdjDiffusion {
  static constexpr int NDIM = KIND == kDiff7 ? 3 : 2;
  static constexpr int R = KIND == kStar9r2 ? 2 : 1;
  static constexpr int NF = 1;
  static constexpr bool REDUCES = true, STAR = true;
  Coef c;
  const T* ut;
  template <class C, class A>
  __device__ __forceinline__ void operator()(const A& U, C (&o)[1], C& red) const {
    C l = U(0, 0, 0, 0);
    C lt;  // (L^T lambda) at the local element
    if (KIND == kJacobi5) {
      C nb = add(add(U(0, 1, 0, 0), U(0, -1, 0, 0)), add(U(0, 0, 1, 0), U(0, 0, -1, 0)));
      lt = fma_(C(-4), l, nb);
    } else if (KIND == kDiff7) {
      C nb = add(add(add(U(0, 1, 0, 0), U(0, -1, 0, 0)), add(U(0, 0, 1, 0), U(0, 0, -1, 0))),
                 add(U(0, 0, 0, 1), U(0, 0, 0, -1)));
      lt = fma_(C(-6), l, nb);
    } else {
      C s1 = add(add(U(0, 1, 0, 0), U(0, -1, 0, 0)), add(U(0, 0, 1, 0), U(0, 0, -1, 0)));
      C s2 = add(add(U(0, 2, 0, 0), U(0, -2, 0, 0)), add(U(0, 0, 2, 0), U(0, 0, -2, 0)));
      lt = fma_(C(4.0 / 3.0), s1, fma_(C(-1.0 / 12.0), s2, mul(C(-5), l)));
    }
    o[0] = fma_(c.get(C()), lt, l);
    red = fma_(lt, ldc(ut + U.gidx(), C()), red);
  }
};

// One later stage of a multi-stage (Runge-Kutta) step: out = a * base + b *
// E(in), where E is the wrapped local function (one forward-Euler step), `in`
// the previous stage's state (read with its halo) and `base` the state at the
// start of the step, read only at the local element.  Because base is read
// only where the stage writes, it may be the stage's own output buffer.
template <class Op, class T>
struct OpStage {
  static constexpr int NDIM = Op::NDIM, R = Op::R, NF = Op::NF;
  static constexpr bool REDUCES = false, STAR = Op::STAR;
  Op op;
  Coef a, b;
  const T* base[kMaxFields];
  template <class C, class A>
  __device__ __forceinline__ void operator()(const A& U, C (&o)[NF], C& red) const {
    C e[NF];
    op(U, e, red);
    const int64_t g = U.gidx();
#pragma unroll
    for (int f = 0; f < NF; ++f) o[f] = fma_(b.get(C()), e[f], mul(a.get(C()), ldc(base[f] + g, C())));
  }
};

}  // namespace lope
