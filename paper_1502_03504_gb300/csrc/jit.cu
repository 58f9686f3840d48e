// Local functions written by the user as source and compiled at run time.
//
// The paper's programmer writes a CONCURRENT procedure in the LOPe index
// notation and a source-to-source compiler turns it into device kernels (Sec.
// 2.2, Sec. 4).  Here the user gives the body of the local function as C++
// text that reads U(f, dx, dy[, dz]) and writes out[f]; NVRTC compiles it,
// wrapped in a functor with the builtins' interface, into the same kernel
// templates the builtins use (TMA tiles / z-march, trapezoid tiles, direct
// kernel, and their Runge-Kutta stage forms), straight to sm_103a code.  The
// kernel templates reach NVRTC as embedded copies of the device headers
// (generated into the build by build.py), so nothing outside the library is
// read at run time except the CUDA toolkit's own headers (cuda_bf16.h).
//
// NVRTC is loaded with dlopen and the driver through the runtime's entry-point
// query, so the library still loads on hosts without either; a source
// stencil then fails with LOPE_ERR_UNSUPPORTED.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "generic_kernels.cuh"
#include "tma_kernels.cuh"

namespace lope {

// Embedded device headers (generated file, see build.py).
extern const int kJitHeaderCount;
extern const char* const kJitHeaderNames[];
extern const char* const kJitHeaderTexts[];

namespace {

// ------------------------------------------------------------------ NVRTC
struct Nvrtc {
  bool ok = false;
  std::string why;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcAddNameExpression) add_name = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcGetLoweredName) lowered = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

const Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    void* h = nullptr;
    for (const char* name : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"}) {
      h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
      if (h) break;
    }
    if (!h) {
      n.why = "NVRTC (libnvrtc.so.13) is not available";
      return;
    }
#define LOPE_SYM(field, sym)                                           \
  n.field = reinterpret_cast<decltype(n.field)>(dlsym(h, #sym));       \
  if (!n.field) {                                                      \
    n.why = "NVRTC lacks " #sym;                                        \
    return;                                                            \
  }
    LOPE_SYM(create, nvrtcCreateProgram)
    LOPE_SYM(add_name, nvrtcAddNameExpression)
    LOPE_SYM(compile, nvrtcCompileProgram)
    LOPE_SYM(log_size, nvrtcGetProgramLogSize)
    LOPE_SYM(log, nvrtcGetProgramLog)
    LOPE_SYM(cubin_size, nvrtcGetCUBINSize)
    LOPE_SYM(cubin, nvrtcGetCUBIN)
    LOPE_SYM(lowered, nvrtcGetLoweredName)
    LOPE_SYM(destroy, nvrtcDestroyProgram)
#undef LOPE_SYM
    n.ok = true;
  });
  return n;
}

// Directory holding cuda_bf16.h for NVRTC: $CUDA_HOME/include, else the
// toolkit's default location.
std::string cuda_include_dir() {
  for (const char* env : {"LOPE_CUDA_INCLUDE", "CUDA_HOME", "CUDA_PATH"}) {
    const char* v = std::getenv(env);
    if (!v || !*v) continue;
    std::string d(v);
    if (std::strcmp(env, "LOPE_CUDA_INCLUDE") != 0) d += "/include";
    return d;
  }
  return "/usr/local/cuda/include";
}

// ------------------------------------------------------------------ driver API
struct Driver {
  bool ok = false;
  CUresult (*load)(CUmodule*, const void*) = nullptr;
  CUresult (*get_fn)(CUfunction*, CUmodule, const char*) = nullptr;
  CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                     unsigned, CUstream, void**, void**) = nullptr;
  CUresult (*set_attr)(CUfunction, CUfunction_attribute, int) = nullptr;
  CUresult (*occupancy)(int*, CUfunction, int, size_t) = nullptr;
};

const Driver& driver() {
  static Driver d;
  static std::once_flag once;
  std::call_once(once, [] {
    auto get = [](const char* name, int ver, void** p) {
      cudaDriverEntryPointQueryResult q;
      return cudaGetDriverEntryPointByVersion(name, p, ver, cudaEnableDefault, &q) == cudaSuccess &&
             q == cudaDriverEntryPointSuccess;
    };
    void* p[5] = {};
    if (!get("cuModuleLoadData", 12000, &p[0]) || !get("cuModuleGetFunction", 12000, &p[1]) ||
        !get("cuLaunchKernel", 12000, &p[2]) || !get("cuFuncSetAttribute", 12000, &p[3]) ||
        !get("cuOccupancyMaxActiveBlocksPerMultiprocessor", 12000, &p[4]))
      return;
    d.load = reinterpret_cast<decltype(d.load)>(p[0]);
    d.get_fn = reinterpret_cast<decltype(d.get_fn)>(p[1]);
    d.launch = reinterpret_cast<decltype(d.launch)>(p[2]);
    d.set_attr = reinterpret_cast<decltype(d.set_attr)>(p[3]);
    d.occupancy = reinterpret_cast<decltype(d.occupancy)>(p[4]);
    d.ok = true;
  });
  return d;
}

const char* type_name(int dtype) {
  return dtype == kF64 ? "double" : dtype == kF32 ? "float" : "__nv_bfloat16";
}

// ------------------------------------------------------------------ kernel names
// Host mirror of the run-time compiled functor: the same data members (the
// parameters), so that kernel parameter structs have the same layout on both
// sides; the operator exists only in the compiled source.
template <int ND, int RR, int NFF, bool ST>
struct UserOpHost {
  static constexpr int NDIM = ND, R = RR, NF = NFF;
  static constexpr bool REDUCES = false, STAR = ST;
  Coef p[kUserParams];
  int* err;
};

enum : int { kDirectPlain = 0, kDirectStage = 1, kTrapPlain = 2, kTrapRk = 3, kNumKernels = 4 };

// Name expression of kernel `which` for the compiled functor, with the tile
// constants of the host-side shape (TmaShape) so that both sides agree.
template <class T, int RANK, int R, int NF, bool TALL>
std::string tma_name(bool stage, bool wrap) {
  constexpr bool PAIR = tma_pair<T, R>(false);
  using Sh = TmaShape<T, RANK, R, NF, PAIR, TALL>;
  const std::string t = std::is_same<T, float>::value ? "float"
                        : std::is_same<T, double>::value ? "double" : "__nv_bfloat16";
  const std::string op = stage ? "lope::OpStage<lope::UserOp, " + t + ">" : "lope::UserOp";
  char buf[512];
  std::snprintf(buf, sizeof(buf), "&lope::tma%dd_kernel<%s, %s, %d, %d, %d, %d, %s, %s>", RANK,
                op.c_str(), t.c_str(), Sh::TX, Sh::TY, Sh::RY, Sh::S, wrap ? "true" : "false",
                PAIR ? "true" : "false");
  return buf;
}

}  // namespace

// One user-written local function: its source, shape and parameters, the
// compiled code per storage type and the loaded kernels per device.
struct JitProgram {
  std::string body;
  int ndim = 2, radius = 1, nf = 1;
  bool star = true;
  double prm[kUserParams] = {};
  std::mutex mu;
  struct Compiled {
    bool done = false;
    std::string cubin;
    std::vector<std::string> names;    // name expressions, in kernel order
    std::vector<std::string> lowered;  // mangled names, same order
  } code[3];
  struct Loaded {
    CUmodule mod = nullptr;
    std::vector<CUfunction> fn;
    std::vector<int> occ;
    std::vector<size_t> smem;  // dynamic shared memory the function is opted in to
  };
  std::map<std::pair<int, int>, Loaded> loaded;  // (device, dtype)

  bool tma_ok() const { return ndim == 2 || star; }

  std::string source() const {
    std::string s;
    s += "#include \"tma_device.cuh\"\n#include \"generic_device.cuh\"\n";
    s += "namespace lope {\nstruct UserOp {\n";
    s += "  static constexpr int NDIM = " + std::to_string(ndim) + ", R = " + std::to_string(radius) +
         ", NF = " + std::to_string(nf) + ";\n";
    s += std::string("  static constexpr bool REDUCES = false, STAR = ") + (star ? "true" : "false") + ";\n";
    s += "  Coef p[" + std::to_string(kUserParams) + "];\n";
    s += "  int* err;\n";
    s += "  template <class C, class A>\n";
    s += "  __device__ __forceinline__ void operator()(const A& lope_acc, C (&out)[NF], C&) const {\n";
    // A read outside the declared halo (or a corner read by a function
    // declared star-shaped) breaks the no-out-of-bounds rule of Sec. 3.5:
    // literal offsets are refused when the stencil is created; a computed one
    // records kErrHalo in the device error flag (reported by lope_sync_status)
    // and is clamped, so no kernel reads outside its staged tile.  With literal
    // offsets the check folds away at compile time.
    s += "    auto U = [&](int f, int dx, int dy, int dz = 0) -> C {\n";
    s += "      const bool bad = f < 0 || f >= NF || dx < -R || dx > R || dy < -R || dy > R ||\n";
    s += "                       (NDIM == 2 ? dz != 0 : (dz < -R || dz > R)) ||\n";
    s += "                       (STAR && ((dx != 0) + (dy != 0) + (dz != 0) > 1));\n";
    s += "      if (bad) {\n";
    s += "        raise_error(err, kErrHalo);\n";
    s += "        f = f < 0 ? 0 : (f >= NF ? NF - 1 : f);\n";
    s += "        dx = dx < -R ? -R : (dx > R ? R : dx);\n";
    s += "        dy = dy < -R ? -R : (dy > R ? R : dy);\n";
    s += "        dz = NDIM == 2 ? 0 : (dz < -R ? -R : (dz > R ? R : dz));\n";
    s += "        if (STAR && (dx != 0) + (dy != 0) + (dz != 0) > 1) dx = dy = dz = 0;\n";
    s += "      }\n";
    s += "      return lope_acc(f, dx, dy, dz);\n    };\n";
    s += "    C P[" + std::to_string(kUserParams) + "];\n";
    s += "    for (int i = 0; i < " + std::to_string(kUserParams) + "; ++i) P[i] = p[i].get(C());\n";
    s += "    (void)P;\n";
    s += "#line 1 \"local_function\"\n";
    s += body;
    s += "\n  }\n};\n}  // namespace lope\n";
    return s;
  }
};

namespace {

template <class T, int RANK, int R, int NF>
void kernel_names(const JitProgram& jp, std::vector<std::string>* names) {
  names->assign(kNumKernels, std::string());
  const std::string t = type_name(std::is_same<T, float>::value ? kF32
                                  : std::is_same<T, double>::value ? kF64 : kBF16);
  (void)jp;  // the TMA instances are appended by all_names
  (*names)[kDirectPlain] = "&lope::direct_kernel<lope::UserOp, " + t + ">";
  (*names)[kDirectStage] = "&lope::direct_kernel<lope::OpStage<lope::UserOp, " + t + ">, " + t + ">";
  if (RANK == 2) {
    (*names)[kTrapPlain] = "&lope::trap2d_kernel<lope::UserOp, " + t + ">";
    (*names)[kTrapRk] = "&lope::trap2d_rk_kernel<lope::UserOp, " + t + ">";
  }
}

// The TMA kernels come in eight instances: plain or combining stage, with or
// without the halo-wrap code, tall or short tiles; they follow the fixed list
// at kNumKernels + tma_index(stage, wrap, tall).  The two-sweep kernels
// follow at tb2_index(wrap): the 3D march with block-shared u1 planes
// (wrap false), or the 2D tiles without / with the halo-wrap code.
constexpr int tma_index(bool stage, bool wrap, bool tall) {
  return kNumKernels + (stage ? 4 : 0) + (wrap ? 2 : 0) + (tall ? 1 : 0);
}
constexpr int tb2_index(bool wrap) { return kNumKernels + 8 + (wrap ? 1 : 0); }
// The z-march with planes copied by producer warps (ca3d_kernel, tall tiles)
// follows at march_index(): 3D star functions of one field with FP32 / FP64
// storage, for grids whose rows TMA cannot stage.
constexpr int march_index() { return kNumKernels + 10; }
template <class T, int RANK, int NF>
constexpr bool jit_march() {
  return RANK == 3 && NF == 1 && !std::is_same<T, __nv_bfloat16>::value;
}

// Whether the two-sweep kernels are compiled for the program: FP32 / BF16
// storage, star functions of one field and radius 1 in 3D, functions of
// radius 1 or 2 in 2D (box functions included).  The 2D tiles of several fields take 2 rows per consumer warp, as
// the builtins' do.
template <class T, int RANK, int R, int NF>
constexpr bool jit_tb2(bool star) {
  return !std::is_same<T, double>::value && (RANK == 3 ? star && R == 1 && NF == 1 : R <= 2);
}
template <int NF> constexpr int jit_tb2_ry() { return NF == 1 ? 8 : 2; }
// (The builtins' box functions of several fields take 4 rows per warp; the
// run-time compiled ones keep one layout, 2 rows, for every function.)

template <class T, int RANK, int R, int NF>
void all_names(const JitProgram& jp, std::vector<std::string>* names) {
  kernel_names<T, RANK, R, NF>(jp, names);
  names->resize(kNumKernels + 11);
  if (!jp.tma_ok()) return;
  if constexpr (jit_march<T, RANK, NF>()) {
    using CR = CaRunner<UserOpHost<RANK, R, NF, true>, T>;
    using S_ = typename CR::template Sh<true>;
    char buf[256];
    std::snprintf(buf, sizeof(buf), "&lope::ca3d_kernel<lope::UserOp, %s, %d, %d, %d, %d, %s, %d>",
                  std::is_same<T, float>::value ? "float" : "double", S_::TX, S_::TY, S_::RY,
                  CR::template stages<true>(), CR::PAIR ? "true" : "false", CR::NPW);
    (*names)[march_index()] = buf;
  }
  for (int stage = 0; stage < 2; ++stage)
    for (int wrap = 0; wrap < 2; ++wrap) {
      (*names)[tma_index(stage, wrap, true)] = tma_name<T, RANK, R, NF, true>(stage, wrap);
      (*names)[tma_index(stage, wrap, false)] = tma_name<T, RANK, R, NF, false>(stage, wrap);
    }
  if constexpr (jit_tb2<T, RANK, R, NF>(true)) {
    if (!jit_tb2<T, RANK, R, NF>(jp.star)) return;
    const std::string t = type_name(std::is_same<T, float>::value ? kF32 : kBF16);
    char buf[256];
    if constexpr (RANK == 3) {
      using Sh = Tb2sShape<T>;
      std::snprintf(buf, sizeof(buf), "&lope::tma3d_tb2s_kernel<lope::UserOp, %s, %d, %d, %d, %d>",
                    t.c_str(), Sh::TX, Sh::TY, Sh::RY, Sh::S);
      (*names)[tb2_index(false)] = buf;
    } else {
      using Sh = Tb2Shape2D<T, R, jit_tb2_ry<NF>(), NF>;
      for (int wrap = 0; wrap < 2; ++wrap) {
        std::snprintf(buf, sizeof(buf), "&lope::tma2d_tb2_kernel<lope::UserOp, %s, %d, %d, %d, %s>",
                      t.c_str(), Sh::TY, Sh::RY, Sh::S, wrap ? "true" : "false");
        (*names)[tb2_index(wrap)] = buf;
      }
    }
  }
}

// Dispatch a functor template over the run-time shape (storage type, rank,
// radius, fields) to the compile-time instance.
template <class F>
auto with_shape(int dtype, int ndim, int radius, int nf, F&& f) {
  auto by_t = [&](auto tag) {
    using T = decltype(tag);
    auto by_rank = [&](auto rank_tag) {
      constexpr int RANK = decltype(rank_tag)::value;
      auto by_r = [&](auto r_tag) {
        constexpr int R = decltype(r_tag)::value;
        static_assert(R == 1 || R == 2, "radius");
        switch (nf) {
          case 1: return f(T(), rank_tag, r_tag, std::integral_constant<int, 1>());
          case 2: return f(T(), rank_tag, r_tag, std::integral_constant<int, 2>());
          default: return f(T(), rank_tag, r_tag, std::integral_constant<int, 3>());
        }
      };
      static_assert(RANK == 2 || RANK == 3, "rank");
      return radius == 1 ? by_r(std::integral_constant<int, 1>()) : by_r(std::integral_constant<int, 2>());
    };
    return ndim == 2 ? by_rank(std::integral_constant<int, 2>()) : by_rank(std::integral_constant<int, 3>());
  };
  if (dtype == kF32) return by_t(float());
  if (dtype == kF64) return by_t(double());
  return by_t(__nv_bfloat16());
}

lope_status compile_locked(JitProgram& jp, int dtype, std::string* err) {
  JitProgram::Compiled& c = jp.code[dtype];
  if (c.done) return LOPE_OK;
  const Nvrtc& nv = nvrtc();
  if (!nv.ok) {
    *err = nv.why;
    return LOPE_ERR_UNSUPPORTED;
  }
  std::vector<std::string> names;
  with_shape(dtype, jp.ndim, jp.radius, jp.nf, [&](auto t, auto rank, auto r, auto nf) {
    using T = decltype(t);
    all_names<T, decltype(rank)::value, decltype(r)::value, decltype(nf)::value>(jp, &names);
    return 0;
  });
  const std::string src = jp.source();
  nvrtcProgram prog = nullptr;
  if (nv.create(&prog, src.c_str(), "local_function.cu", kJitHeaderCount, kJitHeaderTexts,
                kJitHeaderNames) != NVRTC_SUCCESS) {
    *err = "nvrtcCreateProgram failed";
    return LOPE_ERR_ALLOC;
  }
  for (const auto& n : names)
    if (!n.empty()) nv.add_name(prog, n.c_str());
  const std::string inc = "-I" + cuda_include_dir();
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=false",
                        "-default-device", inc.c_str()};
  const nvrtcResult rc = nv.compile(prog, 5, opts);
  size_t ls = 0;
  nv.log_size(prog, &ls);
  std::string log(ls, '\0');
  if (ls) nv.log(prog, &log[0]);
  if (rc != NVRTC_SUCCESS) {
    *err = "local function does not compile:\n" + log;
    nv.destroy(&prog);
    return LOPE_ERR_INVALID;
  }
  size_t cs = 0;
  nv.cubin_size(prog, &cs);
  c.cubin.assign(cs, '\0');
  nv.cubin(prog, &c.cubin[0]);
  c.names = names;
  c.lowered.assign(names.size(), std::string());
  for (size_t i = 0; i < names.size(); ++i) {
    if (names[i].empty()) continue;
    const char* lw = nullptr;
    if (nv.lowered(prog, names[i].c_str(), &lw) == NVRTC_SUCCESS && lw) c.lowered[i] = lw;
  }
  nv.destroy(&prog);
  c.done = true;
  return LOPE_OK;
}

// The kernel `which` of the program for the grid's storage type on the
// current device (compiling and loading on first use).
cudaError_t get_kernel(JitProgram& jp, int dtype, int which, size_t smem, int threads,
                       CUfunction* fn, int* occ) {
  std::lock_guard<std::mutex> lk(jp.mu);
  std::string err;
  if (compile_locked(jp, dtype, &err) != LOPE_OK) {
    lope_fail_external(LOPE_ERR_INVALID, err.c_str());
    return cudaErrorInvalidSource;
  }
  const Driver& d = driver();
  if (!d.ok) return cudaErrorNotSupported;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaFree(nullptr)) != cudaSuccess) return e;  // the device's primary context is current
  JitProgram::Loaded& ld = jp.loaded[{dev, dtype}];
  const JitProgram::Compiled& c = jp.code[dtype];
  if (!ld.mod) {
    if (d.load(&ld.mod, c.cubin.data()) != CUDA_SUCCESS) return cudaErrorInvalidKernelImage;
    ld.fn.assign(c.lowered.size(), nullptr);
    ld.occ.assign(c.lowered.size(), -1);
    ld.smem.assign(c.lowered.size(), 48 * 1024);
  }
  if (which >= int(c.lowered.size()) || c.lowered[which].empty()) return cudaErrorNotSupported;
  if (!ld.fn[which]) {
    CUfunction f = nullptr;
    if (d.get_fn(&f, ld.mod, c.lowered[which].c_str()) != CUDA_SUCCESS) return cudaErrorSymbolNotFound;
    ld.fn[which] = f;
  }
  // Opt in to the launch's dynamic shared memory when it exceeds what the
  // function is set for (the trapezoid's window grows with tile and depth).
  if (smem > ld.smem[which]) {
    if (d.set_attr(ld.fn[which], CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, int(smem)) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
    ld.smem[which] = smem;
    ld.occ[which] = -1;
  }
  *fn = ld.fn[which];
  if (occ) {
    if (ld.occ[which] < 0) {
      int o = 0;
      if (d.occupancy(&o, *fn, threads, smem) != CUDA_SUCCESS) o = 1;
      ld.occ[which] = o > 0 ? o : 1;
    }
    *occ = ld.occ[which];
  }
  return cudaSuccess;
}

cudaError_t launch(CUfunction fn, int blocks, int threads, size_t smem, cudaStream_t st,
                   void** args) {
  const CUresult r = driver().launch(fn, unsigned(blocks), 1, 1, unsigned(threads), 1, 1,
                                     unsigned(smem), reinterpret_cast<CUstream>(st), args, nullptr);
  if (r == CUDA_ERROR_INVALID_VALUE) return cudaErrorInvalidValue;
  if (r != CUDA_SUCCESS) return cudaErrorInvalidConfiguration;  // the launch was rejected
  count_launches(1);
  return cudaSuccess;
}

template <class Op, class T>
void fill_stage(OpStage<Op, T>& st, const StepArgs& a) {
  st.a = a.rk_a;
  st.b = a.rk_b;
  for (int f = 0; f < kMaxFields; ++f) st.base[f] = static_cast<const T*>(a.base[f]);
}

template <class T, int RANK, int R, int NF, bool TALL>
cudaError_t run_tma_t(JitProgram& jp, const StepArgs& a, int dtype) {
  constexpr bool PAIR = tma_pair<T, R>(false);
  using Sh = TmaShape<T, RANK, R, NF, PAIR, TALL>;
  using Host = UserOpHost<RANK, R, NF, true>;
  const bool stage = a.stage >= 2;
  Host op;
  for (int i = 0; i < kUserParams; ++i) op.p[i] = jp.prm[i];
  op.err = a.err;
  auto occ = [&](bool wrap) {
    CUfunction f = nullptr;
    int o = 1;
    if (get_kernel(jp, dtype, tma_index(stage, wrap, TALL), Sh::SMEM, Sh::THREADS, &f, &o) !=
        cudaSuccess)
      o = 1;
    return o;
  };
  auto go = [&](auto& p) -> cudaError_t {
    int blocks = 0;
    Sh::geometry(a, p, &blocks, occ);
    TmaMaps<NF> maps;
    cudaError_t e = Sh::prepare(a, p, maps);
    if (e != cudaSuccess) return e;
    const bool wrap = p.per_x || p.per_y;
    const int which = tma_index(stage, wrap, TALL);
    CUfunction f = nullptr;
    if ((e = get_kernel(jp, dtype, which, Sh::SMEM, Sh::THREADS, &f, nullptr)) != cudaSuccess) return e;
    void* args[] = {&maps, &p};
    return launch(f, blocks, Sh::THREADS, Sh::SMEM, a.stream, args);
  };
  if (stage) {
    TmaParams<OpStage<Host, T>, T> p;
    p.op.op = op;
    fill_stage(p.op, a);
    return go(p);
  }
  TmaParams<Host, T> p;
  p.op = op;
  return go(p);
}

// Two sweeps per launch (tb2_supported decided the grid; the kernels exist
// for the program's shape when jit_tb2 holds).
template <class T, int RANK, int R, int NF>
cudaError_t run_tb2(JitProgram& jp, const StepArgs& a, int dtype) {
  if constexpr (jit_tb2<T, RANK, R, NF>(true)) {
    if (!jit_tb2<T, RANK, R, NF>(jp.star)) return cudaErrorNotSupported;
    using Host = UserOpHost<RANK, R, NF, true>;
    TmaParams<Host, T> p;
    for (int i = 0; i < kUserParams; ++i) p.op.p[i] = jp.prm[i];
    p.op.err = a.err;
    TmaMaps<NF> maps;
    CUfunction f = nullptr;
    int occ = 1, blocks = 0;
    if constexpr (RANK == 3) {
      static_assert(NF == 1, "the 3D two-sweep march takes one field");
      using Sh = Tb2sShape<T>;
      cudaError_t e = get_kernel(jp, dtype, tb2_index(false), Sh::SMEM, Sh::THREADS, &f, &occ);
      if (e != cudaSuccess) return e;
      zmarch_geometry(a.g, p, &blocks, Sh::TX, Sh::TY, occ * sm_count());
      if ((e = Sh::prepare(a, p, maps)) != cudaSuccess) return e;
      void* args[] = {&maps, &p};
      return launch(f, blocks, Sh::THREADS, Sh::SMEM, a.stream, args);
    } else {
      using Sh = Tb2Shape2D<T, R, jit_tb2_ry<NF>(), NF>;
      const bool wrap = a.g.bc[2][0] == kPeriodic || a.g.bc[1][0] == kPeriodic;
      cudaError_t e = get_kernel(jp, dtype, tb2_index(wrap), Sh::SMEM, Sh::THREADS, &f, &occ);
      if (e != cudaSuccess) return e;
      blocks = tb2_2d_geometry<Sh>(a.g, p, occ);
      if ((e = Sh::prepare(a, p, maps)) != cudaSuccess) return e;
      void* args[] = {&maps, &p};
      return launch(f, blocks, Sh::THREADS, Sh::SMEM, a.stream, args);
    }
  } else {
    (void)jp;
    (void)a;
    (void)dtype;
    return cudaErrorNotSupported;
  }
}

template <class T, int RANK, int R, int NF>
cudaError_t run_tma(JitProgram& jp, const StepArgs& a, int dtype) {
  if (a.ksteps == 2) return run_tb2<T, RANK, R, NF>(jp, a, dtype);
  return tma_tall(a) ? run_tma_t<T, RANK, R, NF, true>(jp, a, dtype)
                     : run_tma_t<T, RANK, R, NF, false>(jp, a, dtype);
}

// One sweep on the copied-plane z-march (march_supported decided the grid),
// with the builtins' tiles, ring depth and z-chunk split.
template <class T, int RANK, int R, int NF>
cudaError_t run_march(JitProgram& jp, const StepArgs& a, int dtype) {
  if constexpr (jit_march<T, RANK, NF>()) {
    if (!jp.star || a.stage >= 2 || a.ksteps != 1) return cudaErrorNotSupported;
    using Host = UserOpHost<RANK, R, NF, true>;
    using CR = CaRunner<Host, T>;
    using S_ = typename CR::template Sh<true>;
    constexpr size_t smem = CR::template smem<true>();
    constexpr int threads = CR::template threads<true>();
    CUfunction f = nullptr;
    int occ = 1, blocks = 0, zchunk = 0;
    cudaError_t e = get_kernel(jp, dtype, march_index(), smem, threads, &f, &occ);
    if (e != cudaSuccess) return e;
    if (!march_chunks(a.g, S_::TX, S_::TY, R, occ, &blocks, &zchunk))
      return cudaErrorInvalidConfiguration;
    TmaParams<Host, T> p;
    for (int i = 0; i < kUserParams; ++i) p.op.p[i] = jp.prm[i];
    p.op.err = a.err;
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
    for (int k = 0; k < kMaxFields; ++k) {
      p.in[k] = k < NF ? static_cast<const T*>(a.in[k]) : nullptr;
      p.out[k] = k < NF ? static_cast<T*>(a.out[k]) : nullptr;
    }
    p.partials = nullptr;
    p.err = a.err;
    Geom g = a.g;
    void* args[] = {&g, &p};
    return launch(f, blocks, threads, smem, a.stream, args);
  } else {
    (void)jp;
    (void)a;
    (void)dtype;
    return cudaErrorNotSupported;
  }
}

template <class T, int RANK, int R, int NF>
cudaError_t run_direct(JitProgram& jp, const StepArgs& a, int dtype) {
  using Host = UserOpHost<RANK, R, NF, true>;
  Host op;
  for (int i = 0; i < kUserParams; ++i) op.p[i] = jp.prm[i];
  op.err = a.err;
  const T* in[3] = {nullptr, nullptr, nullptr};
  T* out[3] = {nullptr, nullptr, nullptr};
  for (int f = 0; f < NF; ++f) {
    in[f] = static_cast<const T*>(a.in[f]);
    out[f] = static_cast<T*>(a.out[f]);
  }
  Geom g = a.g;
  double* partials = nullptr;
  const int blocks = direct_grid(a.g);
  CUfunction f = nullptr;
  cudaError_t e;
  if (a.stage >= 2) {
    OpStage<Host, T> st;
    st.op = op;
    fill_stage(st, a);
    if ((e = get_kernel(jp, dtype, kDirectStage, 0, 256, &f, nullptr)) != cudaSuccess) return e;
    void* args[] = {&st, &g, &in[0], &in[1], &in[2], &out[0], &out[1], &out[2], &partials};
    return launch(f, blocks, 256, 0, a.stream, args);
  }
  if ((e = get_kernel(jp, dtype, kDirectPlain, 0, 256, &f, nullptr)) != cudaSuccess) return e;
  void* args[] = {&op, &g, &in[0], &in[1], &in[2], &out[0], &out[1], &out[2], &partials};
  return launch(f, blocks, 256, 0, a.stream, args);
}

template <class T, int RANK, int R, int NF>
cudaError_t run_trap(JitProgram& jp, const StepArgs& a, int dtype) {
  if (RANK != 2) return cudaErrorNotSupported;
  using Host = UserOpHost<RANK, R, NF, true>;
  Host op;
  for (int i = 0; i < kUserParams; ++i) op.p[i] = jp.prm[i];
  op.err = a.err;
  int TX = a.tile_x > 0 ? a.tile_x : 64, TY = a.tile_y > 0 ? a.tile_y : 32;
  int k = std::max(1, a.ksteps);
  int stages = std::max(1, a.s.stages);
  TrapGrid g = trap_grid(a.g);
  const size_t smem = trap_smem_bytes(dtype, NF, TX, TY, R * k * stages, stages);
  const int blocks = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
  const T* in[3] = {nullptr, nullptr, nullptr};
  T* out[3] = {nullptr, nullptr, nullptr};
  for (int f = 0; f < NF; ++f) {
    in[f] = static_cast<const T*>(a.in[f]);
    out[f] = static_cast<T*>(a.out[f]);
  }
  CUfunction f = nullptr;
  cudaError_t e;
  if (stages >= 2) {
    if ((e = get_kernel(jp, dtype, kTrapRk, smem, 256, &f, nullptr)) != cudaSuccess) return e;
    void* args[] = {&op, &g, &in[0], &in[1], &in[2], &out[0], &out[1], &out[2], &TX, &TY, &k, &stages};
    return launch(f, blocks, 256, smem, a.stream, args);
  }
  if ((e = get_kernel(jp, dtype, kTrapPlain, smem, 256, &f, nullptr)) != cudaSuccess) return e;
  void* args[] = {&op, &g, &in[0], &in[1], &in[2], &out[0], &out[1], &out[2], &TX, &TY, &k};
  return launch(f, blocks, 256, smem, a.stream, args);
}

}  // namespace

// ------------------------------------------------------------------ entry points
lope_status jit_create(const char* body, int ndim, int radius, int nf, bool star,
                       const double* prm, int nprm, JitProgram** out) {
  auto* jp = new (std::nothrow) JitProgram;
  if (!jp) return LOPE_ERR_ALLOC;
  jp->body = body;
  jp->ndim = ndim;
  jp->radius = radius;
  jp->nf = nf;
  jp->star = star;
  for (int i = 0; i < nprm && i < kUserParams; ++i) jp->prm[i] = prm[i];
  *out = jp;
  return LOPE_OK;
}

void jit_destroy(JitProgram* jp) { delete jp; }

lope_status jit_compile(JitProgram* jp, int dtype, std::string* err) {
  std::lock_guard<std::mutex> lk(jp->mu);
  return compile_locked(*jp, dtype, err);
}

bool jit_tma_ok(const JitProgram* jp) { return jp->tma_ok(); }

cudaError_t jit_launch(const StepArgs& a, int path) {
  JitProgram* jp = static_cast<JitProgram*>(a.s.jit);
  if (!jp) return cudaErrorInvalidValue;
  const int dtype = a.g.dtype;
  return with_shape(dtype, jp->ndim, jp->radius, jp->nf, [&](auto t, auto rank, auto r, auto nf) {
    using T = decltype(t);
    constexpr int RANK = decltype(rank)::value, R = decltype(r)::value, NF = decltype(nf)::value;
    if (path == kPathTma) return run_tma<T, RANK, R, NF>(*jp, a, dtype);
    if (path == kPathTrap) return run_trap<T, RANK, R, NF>(*jp, a, dtype);
    if (path == kPathMarch) return run_march<T, RANK, R, NF>(*jp, a, dtype);
    return run_direct<T, RANK, R, NF>(*jp, a, dtype);
  });
}

}  // namespace lope
