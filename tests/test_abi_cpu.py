"""C ABI checks that need no GPU: the library builds, loads, exports every
declared entry point, and rejects invalid descriptors before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def fake_addresses(lope):
    """For tests that hand the library fake device addresses (never
    dereferenced): every call that gets past the host-side checks stops at the
    library's first allocation with LOPE_ERR_ALLOC, before any CUDA call, so no
    such call can reach a kernel launch.  Skipped where a CUDA device is
    visible, as a second guard."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("fake device addresses are only handed to the library without a GPU")
    lope.lope_set_option("fail_alloc", 1000000)
    try:
        yield
    finally:
        lope.lope_set_option("fail_alloc", 0)


def _declared():
    names = set()
    with open(os.path.join(ROOT, "include", "lope.h")) as fh:
        text = fh.read()
    for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(lope_[a-z_0-9]+)\s*\(", text, re.M):
        names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for n in ("lope_grid_create", "lope_set_boundary", "lope_apply", "lope_apply_batch",
              "lope_adjoint", "lope_vjp", "lope_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lope):
    lib = ctypes.CDLL(lope.library_path())
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_counter(lope):
    assert "sm_103a" in lope.version()
    assert lope.launch_count() >= 0


def test_grid_validation(lope):
    with pytest.raises(lope.LopeError, match="INVALID"):
        lope.Grid((0, 8))
    with pytest.raises(lope.LopeError, match="INVALID"):
        lope.Grid((8, 8, 8, 8))
    with pytest.raises(lope.LopeError, match="INVALID"):
        lope.Grid((8, 8), halo=5)
    g = lope.Grid((8, 8))
    with pytest.raises(lope.LopeError, match="INVALID"):
        g.set_boundary(axis=2)
    with pytest.raises(lope.LopeError, match="INVALID"):
        g.set_boundary(axis=0, side=0, kind="periodic")


def test_stencil_validation(lope):
    with pytest.raises(lope.LopeError, match="unknown builtin"):
        lope.Stencil.builtin("laplace9", 0.1)
    with pytest.raises(lope.LopeError, match="parameter count"):
        lope.Stencil.builtin("swe_cgrid", 0.1)
    with pytest.raises(lope.LopeError):
        lope.Stencil.linear(np.zeros((7, 7)))


def test_halo_bound_is_enforced_before_any_cuda_call(lope, fake_addresses):
    """A radius-2 local function on a halo-1 grid would read out of bounds (Sec. 3.5)."""
    g = lope.Grid((16, 16), halo=1)
    s = lope.Stencil.builtin("star9r2", 0.1)
    with pytest.raises(lope.LopeError, match="halo"):
        lope.lope_apply(g.handle, s.handle, [16], [32], None, 1, None)
    g3 = lope.Grid((4, 4, 4), halo=1)
    with pytest.raises(lope.LopeError, match="dimensions"):
        lope.lope_apply(g3.handle, s.handle, [16], [32], None, 1, None)


def test_field_count_mismatch(lope, fake_addresses):
    g = lope.Grid((16, 16), halo=1, nfields=1)
    s = lope.Stencil.builtin("swe_cgrid", 0.02, 1.0, 1.0)
    with pytest.raises(lope.LopeError, match="field"):
        lope.lope_apply(g.handle, s.handle, [16], [32], None, 1, None)


def test_periodic_axis_shorter_than_radius(lope, fake_addresses):
    g = lope.Grid((1, 16), halo=2)
    s = lope.Stencil.builtin("star9r2", 0.1)
    with pytest.raises(lope.LopeError, match="periodic axis"):
        lope.lope_apply(g.handle, s.handle, [16], [32], None, 1, None)


def test_set_option_validation(lope):
    with pytest.raises(lope.LopeError, match="unknown option"):
        lope.lope_set_option("no_such_option", 1)
    with pytest.raises(lope.LopeError, match="range"):
        lope.lope_set_option("wait_limit_ms", 0)
    lope.lope_set_option("wait_limit_ms", 1000)
    lope.lope_set_option("batch_skip_arrive", -1)
    with pytest.raises(lope.LopeError):
        lope.lope_set_option("log", 2)
    lope.lope_set_option("log", 0)


def test_noalloc_reduce_rejects_bad_arguments_without_gpu(lope):
    with pytest.raises(lope.LopeError, match="2\\^28"):
        lope.lope_reduce_noalloc(0, lope.DTYPES["f32"], 16, 0, (1 << 28) + 1, 32, None)
    with pytest.raises(lope.LopeError, match="bad reduction"):
        lope.lope_reduce_noalloc(7, lope.DTYPES["f32"], 16, 0, 10, 32, None)


def test_apply_arguments_are_checked_before_any_cuda_call(lope, fake_addresses):
    """Misaligned, missing and aliasing buffers fail on the host (fake device
    addresses, never dereferenced), before the library touches CUDA."""
    g = lope.Grid((64, 64), halo=1)  # 16 KiB per FP32 field
    s = lope.Stencil.builtin("jacobi5", 0.2)
    base, field = 1 << 40, 64 * 64 * 4
    with pytest.raises(lope.LopeError, match="16-byte aligned"):
        lope.lope_apply(g.handle, s.handle, [base + 4], [base + 2 * field], None, 1, None)
    with pytest.raises(lope.LopeError, match="aliases"):
        lope.lope_apply(g.handle, s.handle, [base], [base + field // 2], None, 1, None)
    direct = lope.Launch(3, 0, 0, 0, -1)  # one sweep per launch: 3 steps need a work buffer
    with pytest.raises(lope.LopeError, match="work buffers"):
        lope.lope_apply_with(g.handle, s.handle, [base], [base + field], None, 3, direct, None)
    with pytest.raises(lope.LopeError, match="work aliases"):
        lope.lope_apply_with(g.handle, s.handle, [base], [base + field], [base + field + 256], 3,
                             direct, None)
    with pytest.raises(lope.LopeError, match="NULL field"):
        lope.lope_apply(g.handle, s.handle, [0], [base], None, 1, None)
    with pytest.raises(lope.LopeError, match="nsteps"):
        lope.lope_apply(g.handle, s.handle, [base], [base + field], None, -1, None)
    # multi-stage: RK3 on the stage path needs two states per work buffer
    s.set_scheme("rk3")
    with pytest.raises(lope.LopeError, match="work aliases"):
        lope.lope_apply_with(g.handle, s.handle, [base], [base + 2 * field], [base + field], 1,
                             lope.Launch(3, 0, 0, 0, -1), None)
    # a launch path that cannot take the grid is refused by the planner
    g3 = lope.Grid((8, 8, 10), halo=1)  # 40-byte rows: no TMA staging
    s3 = lope.Stencil.builtin("diff7", 0.1)
    with pytest.raises(lope.LopeError, match="does not support"):
        lope.lope_apply_with(g3.handle, s3.handle, [base], [base + 4096], None, 1,
                             lope.Launch(1, 0, 0, 0, -1), None)
    with pytest.raises(lope.LopeError, match="does not support"):
        lope.lope_apply_with(g3.handle, s3.handle, [base], [base + 4096], None, 1,
                             lope.Launch(2, 64, 32, 1, -1), None)


def test_tune_cache_file_round_trip_and_planning(lope, tmp_path, capfd, fake_addresses):
    """A cache file's entries are installed for the named GPU only, written back
    unchanged, and used by the planner (visible in the plan log, which is
    printed before any CUDA call)."""
    gpu = "Test GB300"
    lines = [
        # a 1000 x 256 FP32 jacobi5 grid (extents slowest first; kind 1, radius 1,
        # star), periodic: the direct kernel
        "lope-tune 1 Test_GB300 grid 2 1 1000 256 1 1 1 1 0 1 1 : 3 0 0 1",
        # a batch of two grids: 64 x 16 tiles, depth 2
        "lope-tune 1 Test_GB300 batch 20 2 1 1 1 1 0 0 0 0 0 64 64 0 0 0 0 0 0 0 0 : 2 64 16 2",
    ]
    other = ["lope-tune 1 Other_GPU grid 2 1 8 8 1 1 1 1 0 1 1 : 3 0 0 1",
             "lope-tune 1 Test_GB300 grid 2 1 8 8 1 1 1 1 0 1 1 : 9 0 0 1",  # no such path
             "lope-tune 2 Test_GB300 grid 2 1 8 8 1 1 1 1 0 1 1 : 3 0 0 1",  # unknown version
             "garbage", ""]
    src = tmp_path / "tune.txt"
    src.write_text("\n".join(lines + other) + "\n")
    assert lope.lope_tune_cache_load(src, gpu) == 2
    assert lope.lope_tune_cache_load(src, "Another GPU") == 0
    out = tmp_path / "saved.txt"
    lope.lope_tune_cache_save(out, gpu)
    saved = set(out.read_text().splitlines())
    assert set(lines) <= saved
    # the planner takes the loaded choice for that grid
    g = lope.Grid((1000, 256), halo=1)
    s = lope.Stencil.builtin("jacobi5", 0.2)
    base, field = 1 << 40, 256 * 1000 * 4
    lope.lope_set_option("log", 1)
    try:
        with pytest.raises(lope.LopeError, match="LOPE_ERR_ALLOC"):  # stops before any CUDA call
            lope.lope_apply(g.handle, s.handle, [base], [base + field], None, 1, None)
    finally:
        lope.lope_set_option("log", 0)
    err = capfd.readouterr().err
    assert "grid 1000x256 f32" in err and "path=direct" in err
    with pytest.raises(lope.LopeError, match="open"):
        lope.lope_tune_cache_load(tmp_path / "missing.txt", gpu)


PLAN_CASES = [  # shape, dtype, builtin, params, halo, scheme, bc, expected plan-log fragment
    ((512, 512, 512), "f32", "diff7", [0.1], 1, "euler", [1, 1, 1], "path=tma tile=0x0 k=2"),
    ((256, 256, 256), "f32", "diff7", [0.1], 1, "euler", [0, 0, 0], "path=tma tile=0x0 k=1"),
    ((8192, 8192), "f32", "star9r2", [0.1], 2, "euler", [0, 0], "path=tma tile=0x0 k=2"),
    ((4096, 4096), "bf16", "star9r2", [0.1], 2, "euler", [0, 0], "path=tma tile=0x0 k=2"),
    ((1536, 2048), "f32", "star9r2", [0.1], 2, "euler", [0, 1], "path=tma tile=0x0 k=1"),
    ((256, 256), "f64", "jacobi5", [0.2], 1, "euler", [0, 0], "path=trapezoid tile=64x16 k=4"),
    ((7094, 7094), "f32", "jacobi5", [0.2], 1, "euler", [0, 1], "path=trapezoid tile=128x32 k=4"),
    ((7094, 7094), "f32", "swe_flux", [0.02, 1.0, 0.5, 1.0], 1, "euler", [0, 0],
     "path=trapezoid tile=64x16 k=4"),
    ((130, 500, 510), "f32", "diff7", [0.1], 1, "euler", [1, 0, 1], "path=march"),
    ((8192, 8192), "f32", "jacobi5", [0.2], 1, "rk3", [0, 0], "path=trapezoid tile=128x16 k=1"),
    ((4096, 4096), "f32", "swe_flux", [0.02, 1.0, 0.5, 1.0], 1, "rk3", [0, 0], "path=tma"),
    ((4096, 4096), "f32", "swe_cgrid", [0.02, 1.0, 1.0], 1, "euler", [0, 0], "path=tma tile=0x0 k=2"),
    ((4096, 4096), "bf16", "swe_cgrid", [0.02, 1.0, 1.0], 1, "euler", [0, 0], "path=tma tile=0x0 k=2"),
    ((4096, 4096), "f32", "swe_flux", [0.02, 1.0, 0.5, 1.0], 1, "euler", [0, 0],
     "path=tma tile=0x0 k=2"),
    ((4096, 4096), "bf16", "swe_flux", [0.02, 1.0, 0.5, 1.0], 1, "euler", [0, 0],
     "path=tma tile=0x0 k=1"),
]


@pytest.mark.parametrize("case", PLAN_CASES, ids=lambda c: f"{c[2]}-{'x'.join(map(str, c[0]))}-{c[5]}")
def test_planner_default_choices(lope, capfd, case, fake_addresses):
    """The planner's documented defaults, read from the plan log (printed before
    the first CUDA call; fake device addresses, never dereferenced)."""
    shape, dtype, name, prm, halo, scheme, bc, want = case
    nf = 3 if name.startswith("swe") else 1
    g = lope.Grid(shape, dtype, halo=halo, nfields=nf)
    g.set_boundaries(bc)
    st = lope.Stencil.builtin(name, *prm).set_scheme(scheme)
    esz = {"f32": 4, "f64": 8, "bf16": 2}[dtype]
    field = int(np.prod(shape)) * esz
    base = 1 << 44
    ins = [base + k * field for k in range(nf)]
    outs = [base + (nf + k) * field for k in range(nf)]
    works = [base + (2 * nf + 2 * k) * field for k in range(nf)]
    lope.lope_set_option("log", 1)
    try:
        with pytest.raises(lope.LopeError, match="LOPE_ERR_ALLOC"):  # stops before any CUDA call
            lope.lope_apply(g.handle, st.handle, ins, outs, works, 10, None)
    finally:
        lope.lope_set_option("log", 0)
    err = capfd.readouterr().err
    assert want in err, err
    # the same plan through the query call, which makes no CUDA call at all
    plan, launches = lope.lope_plan(g.handle, st.handle, ins, outs, works, 10)
    names = {1: "tma", 2: "trapezoid", 3: "direct", 4: "march"}
    assert f"path={names[plan.path]}" in want
    if plan.path == 2 or "k=" in want:
        assert f"tile={plan.tile_x}x{plan.tile_y} k={plan.tsteps}" in want
    assert f"launches={launches}" in err


USER_PLAN_CASES = [  # dtype, nfields, box, scheme, expected path on rows TMA cannot stage
    ("f32", 1, False, "euler", "march"),
    ("f64", 1, False, "euler", "march"),
    ("bf16", 1, False, "euler", "direct"),
    ("f32", 1, True, "euler", "direct"),
    ("f32", 1, False, "rk3", "direct"),
    ("f32", 2, False, "euler", "direct"),
]


@pytest.mark.parametrize("case", USER_PLAN_CASES, ids=lambda c: "-".join(map(str, c)))
def test_planner_user_function_on_unaligned_3d_rows(lope, case, fake_addresses):
    """Run-time compiled functions on 3D rows whose pitch TMA cannot stage: the
    copied-plane z-march for one-field star functions with FP32 / FP64 storage
    and plain sweeps, else the direct kernel (plan query only, no CUDA call)."""
    dtype, nf, box, scheme, want = case
    shape = (130, 500, 509)
    body = "\n".join(f"out[{k}] = add(U({k}, 0, 0, 0), mul(P[0], U({k}, 1, 0, 0)));"
                      for k in range(nf))
    g = lope.Grid(shape, dtype, halo=1, nfields=nf)
    g.set_boundaries([1, 0, 1])
    st = lope.Stencil.source(body, ndim=3, radius=1, nfields=nf, params=[0.1], box=box)
    st.set_scheme(scheme)
    field = int(np.prod(shape)) * {"f32": 4, "f64": 8, "bf16": 2}[dtype]
    base = 1 << 44
    ins = [base + k * field for k in range(nf)]
    outs = [base + (nf + k) * field for k in range(nf)]
    works = [base + (2 * nf + 2 * k) * field for k in range(nf)]
    plan, _ = lope.lope_plan(g.handle, st.handle, ins, outs, works, 10)
    assert {3: "direct", 4: "march"}.get(plan.path) == want, plan.path


def test_apply_host_checks_device_buffers_before_copying(lope, fake_addresses):
    """lope_apply_host refuses bad device buffers before it issues any copy (on a
    machine without a GPU the error is the argument's, not a CUDA error)."""
    g = lope.Grid((64, 64), halo=1)
    s = lope.Stencil.builtin("jacobi5", 0.2)
    host_in, host_out = np.zeros((64, 64), np.float32), np.zeros((64, 64), np.float32)
    base, field = 1 << 40, 64 * 64 * 4
    hin, hout = [host_in.ctypes.data], [host_out.ctypes.data]
    with pytest.raises(lope.LopeError, match="aligned"):
        lope.lope_apply_host(g.handle, s.handle, hin, hout, [base], [base + field + 8], None, 1, None)
    with pytest.raises(lope.LopeError, match="aliases"):
        lope.lope_apply_host(g.handle, s.handle, hin, hout, [base], [base], None, 1, None)
    with pytest.raises(lope.LopeError, match="nsteps"):
        lope.lope_apply_host(g.handle, s.handle, hin, hout, [base], [base + field], None, -2, None)
    # a NULL host pointer of a later field is refused before the copies of the
    # earlier fields are issued
    g3 = lope.Grid((64, 64), halo=1, nfields=3)
    s3 = lope.Stencil.builtin("swe_cgrid", 0.02, 1.0, 1.0)
    hin3 = [host_in.ctypes.data, host_in.ctypes.data, 0]
    hout3 = [host_out.ctypes.data] * 3
    din3 = [base + k * field for k in range(3)]
    dout3 = [base + (3 + k) * field for k in range(3)]
    with pytest.raises(lope.LopeError, match="NULL host"):
        lope.lope_apply_host(g3.handle, s3.handle, hin3, hout3, din3, dout3, None, 1, None)


def test_plan_on_tensors(lope):
    import torch

    g = lope.Grid((300, 301), "f32")
    st = lope.Stencil.builtin("jacobi5", 0.2)
    u, o, w = (torch.zeros(300, 301) for _ in range(3))  # addresses only
    plan, launches = lope.plan(g, st, u, o, w, nsteps=10)
    assert (plan.path, plan.tile_x, plan.tile_y, plan.tsteps, launches) == (2, 64, 16, 4, 3)
    plan, launches = lope.plan(g, st, u, o, w, nsteps=10, launch=lope.Launch(3, 0, 0, 0, -1))
    assert (plan.path, launches, plan.graph) == (3, 10, -1)
    with pytest.raises(lope.LopeError, match="aliases"):
        lope.plan(g, st, u, u, w, nsteps=10)


def test_forced_allocation_failure_is_reported_before_cuda(lope):
    """The fail_alloc option makes the next n calls that may allocate fail with
    LOPE_ERR_ALLOC on the host, before any CUDA call (fake device addresses,
    never dereferenced).  That the call after them proceeds normally is checked
    on the GPU (test_gpu_host.py); here no call may get past the injection."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("fake device addresses are only handed to the library without a GPU")
    g = lope.Grid((64, 64), halo=1)
    s = lope.Stencil.builtin("jacobi5", 0.2)
    base, field = 1 << 40, 64 * 64 * 4
    with pytest.raises(lope.LopeError):
        lope.lope_set_option("fail_alloc", -1)
    lope.lope_set_option("fail_alloc", 2)
    try:
        for _ in range(2):
            with pytest.raises(lope.LopeError, match="LOPE_ERR_ALLOC"):
                lope.lope_apply(g.handle, s.handle, [base], [base + field], None, 1, None)
        # a host-side argument error still comes first while failures are pending
        lope.lope_set_option("fail_alloc", 1)
        with pytest.raises(lope.LopeError, match="aligned"):
            lope.lope_apply(g.handle, s.handle, [base + 4], [base + field], None, 1, None)
        with pytest.raises(lope.LopeError, match="LOPE_ERR_ALLOC"):
            lope.lope_apply(g.handle, s.handle, [base], [base + field], None, 1, None)
    finally:
        lope.lope_set_option("fail_alloc", 0)


def test_external_boundary_is_checked_on_the_host(lope, fake_addresses):
    """LOPE_BC_EXTERNAL: slowest axis only, one sweep per call, the TMA or
    direct kernels (planned without any CUDA call; fake device addresses)."""
    g = lope.Grid((64, 64), halo=1)
    with pytest.raises(lope.LopeError, match="slowest axis"):
        g.set_boundary(axis=1, side=0, kind="external")
    g.set_boundaries([(2, 2), 0])
    s = lope.Stencil.builtin("jacobi5", 0.2)
    base, field = 1 << 40, 64 * 64 * 4
    ins, outs, works = [base + 256], [base + 3 * field], [base + 5 * field]
    with pytest.raises(lope.LopeError, match="one sweep per call"):
        lope.lope_plan(g.handle, s.handle, ins, outs, works, 3)
    plan, launches = lope.lope_plan(g.handle, s.handle, ins, outs, None, 1)
    assert (plan.path, launches) == (1, 1)
    with pytest.raises(lope.LopeError, match="UNSUPPORTED"):
        lope.lope_plan(g.handle, s.handle, ins, outs, None, 1, lope.Launch(2, 64, 16, 1, -1))
    # the input's external halo rows count for aliasing: out may not start in them
    with pytest.raises(lope.LopeError, match="aliases"):
        lope.lope_plan(g.handle, s.handle, ins, [base + 256 + field], None, 1)
    # one external side and a Dirichlet value on the other: the direct kernel
    g.set_boundary(axis=0, side=1, kind="dirichlet", value=0.5)
    plan, _ = lope.lope_plan(g.handle, s.handle, ins, outs, None, 1)
    assert plan.path == 3
