"""ctypes binding of liblope.so: argument marshalling only.

Every function here either forwards to the C ABI of ``include/lope.h`` or
allocates torch tensors for it.  No stencil arithmetic happens in Python, and
there is no fallback: if the CUDA library is missing or fails, these calls
raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "liblope.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC = 0
BC_DIRICHLET = 1
BC_EXTERNAL = 2
DTYPES = {"f64": 0, "f32": 1, "bf16": 2}
_ESIZE = {"f64": 8, "f32": 4, "bf16": 2}
_STATUS = {0: "LOPE_OK", 1: "LOPE_ERR_INVALID", 2: "LOPE_ERR_UNSUPPORTED", 3: "LOPE_ERR_CUDA",
           4: "LOPE_ERR_ALLOC", 5: "LOPE_ERR_TIMEOUT", 6: "LOPE_ERR_NUMERIC"}


class LopeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class Launch(ctypes.Structure):
    """lope_launch: path (0 auto, 1 TMA, 2 trapezoid, 3 direct, 4 plane march), tile,
    depth, graph."""

    _fields_ = [("path", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("tsteps", ctypes.c_int), ("graph", ctypes.c_int)]

    def __repr__(self):
        return (f"Launch(path={self.path}, tile_x={self.tile_x}, tile_y={self.tile_y}, "
                f"tsteps={self.tsteps}, graph={self.graph})")


_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_I64 = ctypes.c_int64
_INT = ctypes.c_int
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_SZ = ctypes.c_size_t

_SIGS = {
    "lope_grid_create": (_INT, [ctypes.POINTER(_P), _INT, ctypes.POINTER(_I64),
                                ctypes.POINTER(_INT), ctypes.POINTER(_INT), _INT, _INT]),
    "lope_grid_destroy": (None, [_P]),
    "lope_plan": (_INT, [_P, _P, _PP, _PP, _PP, _I64, ctypes.POINTER(Launch), ctypes.POINTER(Launch),
                         ctypes.POINTER(_I64)]),
    "lope_tune_cache_save": (_INT, [ctypes.c_char_p, ctypes.c_char_p]),
    "lope_tune_cache_load": (_INT, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(_INT)]),
    "lope_set_boundary": (_INT, [_P, _INT, _INT, _INT, _D]),
    "lope_stencil_create_builtin": (_INT, [ctypes.POINTER(_P), ctypes.c_char_p, _DP, _INT]),
    "lope_stencil_create_linear": (_INT, [ctypes.POINTER(_P), _INT, _INT, _DP]),
    "lope_stencil_destroy": (None, [_P]),
    "lope_stencil_set_scheme": (_INT, [_P, _INT]),
    "lope_stencil_create_source": (_INT, [ctypes.POINTER(_P), _INT, _INT, _INT, _INT,
                                          ctypes.c_char_p, _DP, _INT]),
    "lope_stencil_compile": (_INT, [_P, _INT]),
    "lope_work_states": (_INT, [_P, ctypes.POINTER(_INT)]),
    "lope_apply": (_INT, [_P, _P, _PP, _PP, _PP, _I64, _P]),
    "lope_apply_with": (_INT, [_P, _P, _PP, _PP, _PP, _I64, ctypes.POINTER(Launch), _P]),
    "lope_apply_host": (_INT, [_P, _P, _PP, _PP, _PP, _PP, _PP, _I64, _P]),
    "lope_autotune": (_INT, [_P, _P, _PP, _PP, _PP, _I64, ctypes.POINTER(Launch), _DP, _P]),
    "lope_batch_workspace_size": (_INT, [_INT, _PP, _P, ctypes.POINTER(Launch), ctypes.POINTER(_SZ)]),
    "lope_apply_batch": (_INT, [_INT, _PP, _P, _PP, _PP, _PP, _I64, ctypes.POINTER(Launch), _P, _SZ, _P]),
    "lope_autotune_batch": (_INT, [_INT, _PP, _P, _PP, _PP, _PP, _I64, _P, _SZ,
                                   ctypes.POINTER(Launch), _DP, _P]),
    "lope_workspace_size": (_INT, [_P, _P, _I64, _I64, ctypes.POINTER(_SZ)]),
    "lope_forward_ckpt": (_INT, [_P, _P, _P, _P, _I64, _I64, _P, _SZ, _P]),
    "lope_vjp": (_INT, [_P, _P, _P, _P, _I64, _I64, _INT, _P, _P, _P, _SZ, _P]),
    "lope_adjoint": (_INT, [_P, _P, _P, _P, _I64, _I64, _P, _DP, _DP, _P, _SZ, _P]),
    "lope_reduce_scratch_bytes": (_SZ, []),
    "lope_reduce": (_INT, [_INT, _INT, _P, _P, _I64, _P, _P, _P]),
    "lope_reduce_noalloc": (_INT, [_INT, _INT, _P, _P, _I64, _P, _P]),
    "lope_sync_status": (_INT, [_P]),
    "lope_set_option": (_INT, [ctypes.c_char_p, _I64]),
    "lope_launch_count": (_I64, []),
    "lope_last_error": (ctypes.c_char_p, []),
    "lope_version": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return _LIBPATH


def load():
    """Load liblope.so (built by ``paper_1502_03504_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIBPATH):
                raise RuntimeError(
                    f"{_LIBPATH} is missing: build the CUDA library first "
                    "(python -m paper_1502_03504_gb300.build); there is no CPU fallback")
            lib = ctypes.CDLL(_LIBPATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int):
    if rc != 0:
        raise LopeError(rc, load().lope_last_error().decode())


def _ptrs(vals) -> ctypes.Array:
    arr = (_P * len(vals))()
    for i, v in enumerate(vals):
        arr[i] = v
    return arr


def _stream(stream):
    import torch

    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


# ---------------------------------------------------------------- C ABI names
def lope_grid_create(ndim, extents, halo_lo, halo_hi, dtype, nfields):
    h = _P()
    ext = (_I64 * ndim)(*extents)
    lo = (_INT * ndim)(*halo_lo)
    hi = (_INT * ndim)(*halo_hi)
    _check(load().lope_grid_create(ctypes.byref(h), ndim, ext, lo, hi, dtype, nfields))
    return h


def lope_grid_destroy(h):
    load().lope_grid_destroy(h)


def lope_set_boundary(h, axis, side, kind, value):
    _check(load().lope_set_boundary(h, axis, side, kind, float(value)))


def lope_stencil_create_builtin(name: str, params: Sequence[float]):
    h = _P()
    arr = (_D * max(1, len(params)))(*params)
    _check(load().lope_stencil_create_builtin(ctypes.byref(h), name.encode(), arr, len(params)))
    return h


def lope_stencil_create_linear(ndim: int, radius: int, weights):
    h = _P()
    w = np.ascontiguousarray(weights, dtype=np.float64).ravel()
    _check(load().lope_stencil_create_linear(ctypes.byref(h), ndim, radius,
                                             w.ctypes.data_as(_DP)))
    return h


SCHEMES = {"euler": 1, "rk2": 2, "rk3": 3}


def lope_stencil_create_source(ndim: int, radius: int, nfields: int, box: bool, body: str,
                               params: Sequence[float] = ()):
    h = _P()
    arr = (ctypes.c_double * max(1, len(params)))(*[float(p) for p in params])
    _check(load().lope_stencil_create_source(ctypes.byref(h), int(ndim), int(radius),
                                             int(nfields), int(bool(box)), body.encode(), arr,
                                             len(params)))
    return h


def lope_stencil_compile(h, dtype: str):
    _check(load().lope_stencil_compile(h, DTYPES[dtype]))


def lope_stencil_set_scheme(h, scheme: int):
    _check(load().lope_stencil_set_scheme(h, int(scheme)))


def lope_work_states(h) -> int:
    n = _INT(0)
    _check(load().lope_work_states(h, ctypes.byref(n)))
    return int(n.value)


def lope_stencil_destroy(h):
    load().lope_stencil_destroy(h)


def lope_apply(grid, stencil, ins, outs, works, nsteps, stream):
    _check(load().lope_apply(grid, stencil, _ptrs(ins), _ptrs(outs),
                             _ptrs(works) if works is not None else None, int(nsteps), stream))


def lope_apply_with(grid, stencil, ins, outs, works, nsteps, launch, stream):
    _check(load().lope_apply_with(grid, stencil, _ptrs(ins), _ptrs(outs),
                                  _ptrs(works) if works is not None else None, int(nsteps),
                                  ctypes.byref(launch) if launch is not None else None, stream))


def lope_autotune(grid, stencil, ins, outs, works, nsteps, stream):
    best = Launch()
    ms = _D()
    _check(load().lope_autotune(grid, stencil, _ptrs(ins), _ptrs(outs), _ptrs(works), int(nsteps),
                                ctypes.byref(best), ctypes.byref(ms), stream))
    return best, ms.value


def lope_batch_workspace_size(grids, stencil, launch=None):
    n = _SZ()
    _check(load().lope_batch_workspace_size(len(grids), _ptrs(grids), stencil,
                                            ctypes.byref(launch) if launch is not None else None,
                                            ctypes.byref(n)))
    return n.value


def lope_apply_batch(grids, stencil, ins, outs, works, nsteps, launch, ws, ws_bytes, stream):
    _check(load().lope_apply_batch(len(grids), _ptrs(grids), stencil, _ptrs(ins), _ptrs(outs),
                                   _ptrs(works), int(nsteps),
                                   ctypes.byref(launch) if launch is not None else None, ws,
                                   ws_bytes, stream))


def lope_workspace_size(grid, stencil, nsteps, ckpt):
    n = _SZ()
    _check(load().lope_workspace_size(grid, stencil, int(nsteps), int(ckpt), ctypes.byref(n)))
    return n.value


def lope_forward_ckpt(grid, stencil, u0, uT, nsteps, ckpt, ws, ws_bytes, stream):
    _check(load().lope_forward_ckpt(grid, stencil, u0, uT, int(nsteps), int(ckpt), ws, ws_bytes,
                                    stream))


def lope_vjp(grid, stencil, u0, grad_uT, nsteps, ckpt, reuse, grad_u0, gc_dev, ws, ws_bytes, stream):
    _check(load().lope_vjp(grid, stencil, u0, grad_uT, int(nsteps), int(ckpt), int(reuse), grad_u0,
                           gc_dev, ws, ws_bytes, stream))


def lope_adjoint(grid, stencil, u0, target, nsteps, ckpt, grad_u0, ws, ws_bytes, stream):
    gc = _D()
    loss = _D()
    _check(load().lope_adjoint(grid, stencil, u0, target, int(nsteps), int(ckpt), grad_u0,
                               ctypes.byref(gc), ctypes.byref(loss), ws, ws_bytes, stream))
    return loss.value, gc.value


def lope_reduce_scratch_bytes():
    return int(load().lope_reduce_scratch_bytes())


def lope_reduce(op, dtype, x, y, n, result_dev, scratch, stream):
    _check(load().lope_reduce(op, dtype, x, y, int(n), result_dev, scratch, stream))


def lope_set_option(name: str, value: int):
    _check(load().lope_set_option(name.encode(), int(value)))


def lope_reduce_noalloc(op, dtype, x, y, n, result_dev, stream):
    """FP64 reduction whose partial sums live in the library's own static
    device array: no scratch buffer from the caller (see include/lope.h)."""
    _check(load().lope_reduce_noalloc(op, dtype, x, y, int(n), result_dev, stream))


def lope_plan(grid, stencil, ins, outs, works, nsteps, launch=None):
    """The plan lope_apply_with would run: (Launch, number of launches)."""
    plan = Launch()
    n = _I64(0)
    _check(load().lope_plan(grid, stencil, _ptrs(ins), _ptrs(outs),
                            _ptrs(works) if works is not None else None, int(nsteps),
                            ctypes.byref(launch) if launch is not None else None,
                            ctypes.byref(plan), ctypes.byref(n)))
    return plan, n.value


def lope_tune_cache_save(path: str, gpu_name=None):
    _check(load().lope_tune_cache_save(str(path).encode(),
                                       gpu_name.encode() if gpu_name is not None else None))


def lope_tune_cache_load(path: str, gpu_name=None) -> int:
    n = _INT(0)
    _check(load().lope_tune_cache_load(str(path).encode(),
                                       gpu_name.encode() if gpu_name is not None else None,
                                       ctypes.byref(n)))
    return n.value


def lope_sync_status(stream):
    _check(load().lope_sync_status(stream))


def lope_launch_count():
    return int(load().lope_launch_count())


def lope_last_error():
    return load().lope_last_error().decode()


def lope_version():
    return load().lope_version().decode()


# ---------------------------------------------------------------- torch helpers
def _torch_dtype(name):
    import torch

    return {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[name]


class Grid:
    """A halo-annotated grid: extents (slowest first), halo widths, dtype, fields."""

    def __init__(self, shape, dtype="f32", halo=1, nfields=1):
        self.shape = tuple(int(s) for s in shape)
        self.ndim = len(self.shape)
        self.dtype = dtype
        self.nfields = nfields
        hl = [halo] * self.ndim if np.isscalar(halo) else list(halo)
        self.handle = lope_grid_create(self.ndim, self.shape, hl, hl, DTYPES[dtype], nfields)

    def set_boundary(self, axis=-1, side=-1, kind="periodic", value=0.0):
        names = {"periodic": BC_PERIODIC, "dirichlet": BC_DIRICHLET, "external": BC_EXTERNAL}
        k = names[kind] if isinstance(kind, str) else int(kind)
        lope_set_boundary(self.handle, axis, side, k, value)
        return self

    def set_boundaries(self, bc, bval=None):
        """bc: list per axis of kind (0 periodic / 1 Dirichlet / 2 external) or
        (low, high); bval likewise."""
        bval = bval if bval is not None else [0.0] * self.ndim
        for ax in range(self.ndim):
            k, v = bc[ax], bval[ax]
            kl, kh = (k, k) if np.isscalar(k) else tuple(k)
            vl, vh = (v, v) if np.isscalar(v) else tuple(v)
            if kl == BC_PERIODIC and kh == BC_PERIODIC:
                lope_set_boundary(self.handle, ax, -1, BC_PERIODIC, 0.0)
            else:
                lope_set_boundary(self.handle, ax, 0, kl, vl)
                lope_set_boundary(self.handle, ax, 1, kh, vh)
        return self

    def empty(self, device="cuda"):
        import torch

        return torch.empty(self.shape, dtype=_torch_dtype(self.dtype), device=device)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.lope_grid_destroy(h)
            self.handle = None


class Stencil:
    """A local function: a builtin by name, or a linear weight table."""

    def __init__(self, handle, ndim, radius, nfields):
        self.handle, self.ndim, self.radius, self.nfields = handle, ndim, radius, nfields
        self.scheme = "euler"

    def set_scheme(self, scheme: str):
        """Time-stepping scheme: "euler" (the local function is the step), "rk2", "rk3"."""
        lope_stencil_set_scheme(self.handle, SCHEMES[scheme])
        self.scheme = scheme
        return self

    def work_states(self) -> int:
        return lope_work_states(self.handle)

    @classmethod
    def builtin(cls, name, *params):
        h = lope_stencil_create_builtin(name, [float(p) for p in params])
        ndim = 3 if name == "diff7" else 2
        radius = 2 if name == "star9r2" else 1
        return cls(h, ndim, radius, 3 if name in ("swe_cgrid", "swe_flux") else 1)

    @classmethod
    def source(cls, body: str, ndim: int = 2, radius: int = 1, nfields: int = 1, params=(),
               box: bool = False):
        """A local function written as C++ source (see lope_stencil_create_source):
        it reads U(f, dx, dy[, dz]) and P[i] and assigns out[f]."""
        h = lope_stencil_create_source(ndim, radius, nfields, box, body, list(params))
        st = cls(h, ndim, radius, nfields)
        st.body = body
        return st

    def compile(self, dtype: str = "f32"):
        """Compile a source stencil's kernels for a storage type now (no GPU needed)."""
        lope_stencil_compile(self.handle, dtype)
        return self

    @classmethod
    def linear(cls, weights):
        w = np.asarray(weights, dtype=np.float64)
        radius = (w.shape[0] - 1) // 2
        return cls(lope_stencil_create_linear(w.ndim, radius, w), w.ndim, radius, 1)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.lope_stencil_destroy(h)
            self.handle = None


def _as_list(x):
    return list(x) if isinstance(x, (list, tuple)) else [x]


def apply(grid: Grid, stencil: Stencil, inputs, out=None, work=None, nsteps=1, launch=None,
          stream=None):
    """Run ``nsteps`` sweeps on device tensors; returns ``out`` (list if multi-field)."""
    import torch

    ins = _as_list(inputs)
    outs = _as_list(out) if out is not None else [torch.empty_like(t) for t in ins]
    if work is not None:
        works = _as_list(work)
    elif nsteps >= 2 or stencil.scheme != "euler":
        ns = stencil.work_states()
        works = [torch.empty((ns,) + tuple(t.shape), dtype=t.dtype, device=t.device) for t in ins]
    else:
        works = None
    s = _stream(stream)
    if launch is None:
        lope_apply(grid.handle, stencil.handle, [_dptr(t) for t in ins], [_dptr(t) for t in outs],
                   [_dptr(t) for t in works] if works is not None else None, nsteps, s)
    else:
        lope_apply_with(grid.handle, stencil.handle, [_dptr(t) for t in ins],
                        [_dptr(t) for t in outs],
                        [_dptr(t) for t in works] if works is not None else None, nsteps, launch, s)
    return outs if isinstance(inputs, (list, tuple)) else outs[0]


def plan(grid: Grid, stencil: Stencil, inputs, out, work=None, nsteps=1, launch=None):
    """The launch plan apply() would run on these tensors: (Launch, launches)."""
    ins, outs = _as_list(inputs), _as_list(out)
    works = _as_list(work) if work is not None else None
    return lope_plan(grid.handle, stencil.handle, [_dptr(t) for t in ins], [_dptr(t) for t in outs],
                     [_dptr(t) for t in works] if works is not None else None, nsteps, launch)


def lope_apply_host(grid, stencil, host_in, host_out, dev_in, dev_out, dev_work, nsteps, stream):
    _check(load().lope_apply_host(grid, stencil, _ptrs(host_in), _ptrs(host_out), _ptrs(dev_in),
                                  _ptrs(dev_out), _ptrs(dev_work) if dev_work is not None else None,
                                  int(nsteps), stream))


def apply_host(grid: Grid, stencil: Stencil, host_in, host_out, dev_in, dev_out, dev_work=None,
               nsteps=1, stream=None):
    """lope_apply_host on tensors: host_in/host_out are (pinned) CPU tensors,
    dev_in/dev_out/dev_work device tensors (lists for multi-field grids)."""
    hi, ho, di, do = (_as_list(x) for x in (host_in, host_out, dev_in, dev_out))
    dw = _as_list(dev_work) if dev_work is not None else None
    lope_apply_host(grid.handle, stencil.handle, [t.data_ptr() for t in hi],
                    [t.data_ptr() for t in ho], [_dptr(t) for t in di], [_dptr(t) for t in do],
                    [_dptr(t) for t in dw] if dw is not None else None, nsteps, _stream(stream))
    return host_out


def autotune(grid, stencil, inputs, out, work, nsteps, stream=None):
    ins, outs, works = _as_list(inputs), _as_list(out), _as_list(work)
    return lope_autotune(grid.handle, stencil.handle, [_dptr(t) for t in ins],
                         [_dptr(t) for t in outs], [_dptr(t) for t in works], nsteps,
                         _stream(stream))


def batch_workspace_size(grids, stencil, launch=None):
    return lope_batch_workspace_size([g.handle for g in grids], stencil.handle, launch)


def apply_batch(grids, stencil, inputs, outs=None, works=None, nsteps=1, launch=None,
                workspace=None, stream=None):
    import torch

    outs = outs if outs is not None else [torch.empty_like(t) for t in inputs]
    works = works if works is not None else [torch.empty_like(t) for t in inputs]
    nb = batch_workspace_size(grids, stencil, launch)
    if workspace is None:
        workspace = torch.empty(nb, dtype=torch.uint8, device=inputs[0].device)
    lope_apply_batch([g.handle for g in grids], stencil.handle, [_dptr(t) for t in inputs],
                     [_dptr(t) for t in outs], [_dptr(t) for t in works], nsteps, launch,
                     _dptr(workspace), workspace.numel(), _stream(stream))
    return outs


def lope_autotune_batch(grids, stencil, ins, outs, works, nsteps, ws, ws_bytes, stream):
    best = Launch()
    ms = ctypes.c_double(0.0)
    _check(load().lope_autotune_batch(len(grids), _ptrs(grids), stencil, _ptrs(ins), _ptrs(outs),
                                      _ptrs(works), int(nsteps), ws, int(ws_bytes),
                                      ctypes.byref(best), ctypes.byref(ms), stream))
    return best, ms.value


def autotune_batch(grids, stencil, inputs, outs, works, nsteps, workspace=None, stream=None):
    """Time the batched launch's tile shapes and depths on these buffers and
    remember the fastest for this batch; returns (Launch, ms)."""
    import torch

    nb = batch_workspace_size(grids, stencil)
    if workspace is None:
        workspace = torch.empty(nb, dtype=torch.uint8, device=inputs[0].device)
    return lope_autotune_batch([g.handle for g in grids], stencil.handle,
                               [_dptr(t) for t in inputs], [_dptr(t) for t in outs],
                               [_dptr(t) for t in works], nsteps, _dptr(workspace),
                               workspace.numel(), _stream(stream))


def workspace_size(grid, stencil, nsteps, ckpt):
    return lope_workspace_size(grid.handle, stencil.handle, nsteps, ckpt)


def _workspace(grid, stencil, nsteps, ckpt, workspace, device):
    import torch

    nb = workspace_size(grid, stencil, nsteps, ckpt)
    if workspace is None or workspace.numel() < nb:
        workspace = torch.empty(nb, dtype=torch.uint8, device=device)
    return workspace


def adjoint(grid, stencil, u0, target, nsteps, ckpt, grad_u0=None, workspace=None, stream=None):
    """(loss, dL/du0, dL/dc) of loss = sum((u_T - target)^2)."""
    import torch

    ws = _workspace(grid, stencil, nsteps, ckpt, workspace, u0.device)
    g = grad_u0 if grad_u0 is not None else torch.empty_like(u0)
    loss, gc = lope_adjoint(grid.handle, stencil.handle, _dptr(u0), _dptr(target), nsteps, ckpt,
                            _dptr(g), _dptr(ws), ws.numel(), _stream(stream))
    return loss, g, gc


def forward_ckpt(grid, stencil, u0, nsteps, ckpt, uT=None, workspace=None, stream=None):
    import torch

    ws = _workspace(grid, stencil, nsteps, ckpt, workspace, u0.device)
    out = uT if uT is not None else torch.empty_like(u0)
    lope_forward_ckpt(grid.handle, stencil.handle, _dptr(u0), _dptr(out), nsteps, ckpt, _dptr(ws),
                      ws.numel(), _stream(stream))
    return out, ws


def vjp(grid, stencil, u0, grad_uT, nsteps, ckpt, reuse=False, workspace=None, stream=None):
    """(dL/du0, dL/dc as a device float64 tensor of shape [1])."""
    import torch

    ws = _workspace(grid, stencil, nsteps, ckpt, workspace, u0.device)
    g = torch.empty_like(u0)
    gc = torch.zeros(1, dtype=torch.float64, device=u0.device)
    lope_vjp(grid.handle, stencil.handle, _dptr(u0), _dptr(grad_uT.contiguous()), nsteps, ckpt,
             1 if reuse else 0, _dptr(g), _dptr(gc), _dptr(ws), ws.numel(), _stream(stream))
    return g, gc


def _reduce(op, x, y=None, stream=None):
    import torch

    name = {torch.float64: "f64", torch.float32: "f32", torch.bfloat16: "bf16"}[x.dtype]
    res = torch.empty(1, dtype=torch.float64, device=x.device)
    scratch = torch.empty(lope_reduce_scratch_bytes(), dtype=torch.uint8, device=x.device)
    lope_reduce(op, DTYPES[name], _dptr(x), _dptr(y), x.numel(), _dptr(res), _dptr(scratch),
                _stream(stream))
    return res


def reduce_sum(x, stream=None):
    """FP64 sum of a field, on the device."""
    return _reduce(0, x, None, stream)


def reduce_sqdiff(x, y, stream=None):
    """FP64 sum of (x - y)^2, on the device."""
    return _reduce(1, x, y, stream)


def sync_status(stream=None):
    lope_sync_status(_stream(stream))


def launch_count():
    return lope_launch_count()


def version():
    return lope_version()
