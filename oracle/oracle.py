"""ctypes binding for oracle/liboracle.so (test infrastructure only).

The arithmetic is in ``lope_oracle.c``; this file marshals numpy arrays.
Boundary specification: ``bc`` is a list with one entry per axis, slowest
first, each either a kind (0 periodic, 1 Dirichlet) applied to both sides or a
pair ``(kind_low, kind_high)``; ``bval`` likewise gives Dirichlet values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

BC_PERIODIC = 0
BC_DIRICHLET = 1
KIND = {"linear": 0, "jacobi5": 1, "diff7": 2, "star9r2": 3, "swe_cgrid": 4, "swe_flux": 5}
# Time-stepping schemes: stages of the strong-stability-preserving Runge-Kutta
# methods built from the local function (1 = the local function itself).
SCHEME_STAGES = {"euler": 1, "rk2": 2, "rk3": 3}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lope_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I = ctypes.POINTER(ctypes.c_int)
_DD = ctypes.POINTER(_D)


def build(force: bool = False) -> str:
    """Compile liblope_oracle with gcc (plain C, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_apply.restype = ctypes.c_int
            lib.oracle_apply.argtypes = [ctypes.c_int, _I64, _I, _D, ctypes.c_int, _D, ctypes.c_int,
                                         _D, _DD, _DD, ctypes.c_int64, ctypes.c_int]
            lib.oracle_apply_rk.restype = ctypes.c_int
            lib.oracle_apply_rk.argtypes = [ctypes.c_int, _I64, _I, _D, ctypes.c_int, _D,
                                            ctypes.c_int, _D, ctypes.c_int, _DD, _DD,
                                            ctypes.c_int64, ctypes.c_int]
            lib.oracle_apply_user.restype = ctypes.c_int
            lib.oracle_apply_user.argtypes = [ctypes.c_int, _I64, _I, _D, ctypes.c_int,
                                              ctypes.c_void_p, _D, ctypes.c_int, _DD, _DD,
                                              ctypes.c_int64, ctypes.c_int]
            lib.oracle_vjp.restype = ctypes.c_int
            lib.oracle_vjp.argtypes = [ctypes.c_int, _I64, _I, _D, ctypes.c_int, _D, ctypes.c_int,
                                       _D, _D, _D, ctypes.c_int64, _D, _D, ctypes.c_int]
            lib.oracle_adjoint.restype = ctypes.c_int
            lib.oracle_adjoint.argtypes = [ctypes.c_int, _I64, _I, _D, ctypes.c_int, _D,
                                           ctypes.c_int, _D, _D, _D, ctypes.c_int64, _D, _D, _D,
                                           ctypes.c_int]
            lib.oracle_weights.restype = ctypes.c_int
            lib.oracle_weights.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_int, _D, _D,
                                           ctypes.c_int]
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _grid_args(shape, bc, bval):
    ndim = len(shape)
    ext = np.asarray(shape, dtype=np.int64)
    if bc is None:
        bc = [BC_PERIODIC] * ndim
    if bval is None:
        bval = [0.0] * ndim
    bcs, bvs = [], []
    for ax in range(ndim):
        k = bc[ax]
        v = bval[ax]
        kl, kh = (k, k) if np.isscalar(k) else tuple(k)
        vl, vh = (v, v) if np.isscalar(v) else tuple(v)
        bcs += [int(kl), int(kh)]
        bvs += [float(vl), float(vh)]
    return ndim, ext, np.asarray(bcs, dtype=np.int32), np.asarray(bvs, dtype=np.float64)


def _stencil_args(kind, params, weights_table):
    k = KIND[kind] if isinstance(kind, str) else int(kind)
    prm = np.asarray(params if params is not None else [0.0], dtype=np.float64)
    if k == KIND["linear"]:
        w = np.ascontiguousarray(weights_table, dtype=np.float64)
        radius = (w.shape[-1] - 1) // 2
    else:
        w = np.zeros(1, dtype=np.float64)
        radius = 0
    return k, prm, np.ascontiguousarray(w.ravel()), radius


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def apply(fields, kind, params=None, nsteps=1, bc=None, bval=None, weights_table=None,
          nthreads=1, scheme="euler"):
    """Apply the local function ``nsteps`` times in FP64.

    ``fields`` is one array or a list of arrays (3 for "swe_cgrid" and
    "swe_flux"), all of the grid's shape (slowest axis first).  Returns arrays
    of the same structure.  ``scheme`` "rk2"/"rk3" takes ``nsteps`` steps of the
    strong-stability-preserving Runge-Kutta method whose stages are sweeps of
    the local function (see oracle_apply_rk).
    """
    lib = _load()
    single = isinstance(fields, np.ndarray)
    fl = [fields] if single else list(fields)
    ins = [np.ascontiguousarray(f, dtype=np.float64) for f in fl]
    shape = ins[0].shape
    ndim, ext, bcs, bvs = _grid_args(shape, bc, bval)
    k, prm, w, radius = _stencil_args(kind, params, weights_table)
    outs = [np.empty_like(a) for a in ins]
    in_arr = (_D * len(ins))(*[_dptr(a) for a in ins])
    out_arr = (_D * len(outs))(*[_dptr(a) for a in outs])
    stages = SCHEME_STAGES[scheme]
    if stages == 1:
        rc = lib.oracle_apply(ndim, ext.ctypes.data_as(_I64), bcs.ctypes.data_as(_I), _dptr(bvs),
                              k, _dptr(prm), radius, _dptr(w), in_arr, out_arr, int(nsteps),
                              int(nthreads))
    else:
        rc = lib.oracle_apply_rk(ndim, ext.ctypes.data_as(_I64), bcs.ctypes.data_as(_I),
                                 _dptr(bvs), k, _dptr(prm), radius, _dptr(w), stages, in_arr,
                                 out_arr, int(nsteps), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_apply rejected its arguments")
    return outs[0] if single else outs


def weights(kind, params=None, ndim=2, weights_table=None):
    """The (2r+1)^ndim weight table the oracle's adjoint scatters with."""
    lib = _load()
    k, prm, w, radius = _stencil_args(kind, params, weights_table)
    out = np.zeros(125, dtype=np.float64)
    r = lib.oracle_weights(k, _dptr(prm), ndim, radius, _dptr(w), _dptr(out), 125)
    if r < 0:
        raise ValueError("no weight table for this stencil")
    side = 2 * r + 1
    shape = (side,) * ndim
    return out[: side ** ndim].reshape(shape).copy()


def vjp(u0, lamT, kind, params=None, nsteps=1, bc=None, bval=None, weights_table=None,
        nthreads=1):
    """(dL/du0, dL/dc) for upstream gradient lamT = dL/du_T (full trajectory)."""
    lib = _load()
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    lamT = np.ascontiguousarray(lamT, dtype=np.float64)
    ndim, ext, bcs, bvs = _grid_args(u0.shape, bc, bval)
    k, prm, w, radius = _stencil_args(kind, params, weights_table)
    g = np.empty_like(u0)
    gc = np.zeros(1, dtype=np.float64)
    rc = lib.oracle_vjp(ndim, ext.ctypes.data_as(_I64), bcs.ctypes.data_as(_I), _dptr(bvs), k,
                        _dptr(prm), radius, _dptr(w), _dptr(u0), _dptr(lamT), int(nsteps),
                        _dptr(g), _dptr(gc), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_vjp rejected its arguments")
    return g, float(gc[0])


def adjoint(u0, target, kind, params=None, nsteps=1, bc=None, bval=None, weights_table=None,
            nthreads=1):
    """(loss, dL/du0, dL/dc) for loss = sum((u_T - target)^2)."""
    lib = _load()
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    target = np.ascontiguousarray(target, dtype=np.float64)
    ndim, ext, bcs, bvs = _grid_args(u0.shape, bc, bval)
    k, prm, w, radius = _stencil_args(kind, params, weights_table)
    g = np.empty_like(u0)
    gc = np.zeros(1, dtype=np.float64)
    loss = np.zeros(1, dtype=np.float64)
    rc = lib.oracle_adjoint(ndim, ext.ctypes.data_as(_I64), bcs.ctypes.data_as(_I), _dptr(bvs),
                            k, _dptr(prm), radius, _dptr(w), _dptr(u0), _dptr(target),
                            int(nsteps), _dptr(g), _dptr(gc), _dptr(loss), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_adjoint rejected its arguments")
    return float(loss[0]), g, float(gc[0])


# ---------------------------------------------------------------- user source
# A local function written as source (the text the library compiles for the
# GPU) is compiled here for the host with g++, in FP64: C is double, U reads
# the oracle's own boundary-aware accessor, and add/sub/mul/fma_ are the plain
# double operations.  The body is the definition; nothing of the GPU path is
# involved.
_USER_PRELUDE = """
namespace {
typedef double C;
inline double add(double a, double b) { return a + b; }
inline double sub(double a, double b) { return a - b; }
inline double mul(double a, double b) { return a * b; }
inline double fma_(double a, double b, double c) { return a * b + c; }
}
extern "C" void lope_user_lf(const void* acc, double (*Uf)(const void*, int, int, int, int),
                             const double* P, double* out) {
  auto U = [&](int f, int dx, int dy, int dz = 0) -> double { return Uf(acc, f, dx, dy, dz); };
  (void)P;
"""
_USER_DIR = os.path.join(_HERE, "_user")
_user_libs = {}


def _user_fn(body: str):
    import hashlib

    key = hashlib.sha256(body.encode()).hexdigest()[:20]
    with _lock:
        if key in _user_libs:
            return _user_libs[key]
        os.makedirs(_USER_DIR, exist_ok=True)
        so = os.path.join(_USER_DIR, f"lf_{key}.so")
        if not os.path.exists(so):
            src = os.path.join(_USER_DIR, f"lf_{key}.{os.getpid()}.cpp")
            with open(src, "w") as fh:
                fh.write(_USER_PRELUDE + "#line 1 \"local_function\"\n" + body + "\n}\n")
            tmp = so + f".tmp{os.getpid()}"
            subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                            src, "-o", tmp], check=True)
            os.replace(tmp, so)
            os.remove(src)
        lib = ctypes.CDLL(so)
        fn = ctypes.cast(lib.lope_user_lf, ctypes.c_void_p).value
        _user_libs[key] = (lib, fn)
        return _user_libs[key]


def apply_source(fields, body, params=(), nsteps=1, bc=None, bval=None, nthreads=1,
                 scheme="euler"):
    """Apply a user-written local function (source text) ``nsteps`` times in FP64."""
    lib = _load()
    _, fn = _user_fn(body)
    single = isinstance(fields, np.ndarray)
    fl = [fields] if single else list(fields)
    ins = [np.ascontiguousarray(f, dtype=np.float64) for f in fl]
    ndim, ext, bcs, bvs = _grid_args(ins[0].shape, bc, bval)
    prm = np.zeros(8, dtype=np.float64)
    prm[: len(params)] = params
    outs = [np.empty_like(a) for a in ins]
    in_arr = (_D * len(ins))(*[_dptr(a) for a in ins])
    out_arr = (_D * len(outs))(*[_dptr(a) for a in outs])
    rc = lib.oracle_apply_user(ndim, ext.ctypes.data_as(_I64), bcs.ctypes.data_as(_I), _dptr(bvs),
                               len(ins), fn, _dptr(prm), SCHEME_STAGES[scheme], in_arr, out_arr,
                               int(nsteps), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_apply_user rejected its arguments")
    return outs[0] if single else outs
