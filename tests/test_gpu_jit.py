"""GPU parity of user-written local functions compiled at run time (NVRTC).

Bodies that spell the builtins with the same operations must give bitwise the
builtins' results on every kernel path (TMA tiles / z-march, trapezoid, direct,
and the Runge-Kutta forms): the same kernel templates run the same arithmetic.
A function with no builtin counterpart (Gray-Scott, two coupled nonlinear
fields) is compared with the oracle, which compiles the same text for the host
in FP64 (FP64: normwise 1e-12; FP32: the bound of gpu_helpers), and across
paths bitwise.
"""
import numpy as np
import pytest
import torch

import lope_inputs as LI
from error_bounds import gray_scott_majorant
from gpu_helpers import normwise, to_device, to_host
from user_bodies import DIFF7, GRAY_SCOTT, GRAY_SCOTT_PRM, JACOBI5, STAR_R2_3D, SWE_FLUX

pytestmark = pytest.mark.gpu

TMA, TRAP, DIRECT, MARCH = 1, 2, 3, 4
FLUX = [0.02, 1.0, 0.5, 1.0]


def _launch(L, path, tx=0, ty=0, k=0, graph=-1):
    return L.Launch(path, tx, ty, k, graph)


def _grid(L, shape, dtype, halo, bc, bval=None, nf=1):
    g = L.Grid(shape, dtype, halo=halo, nfields=nf)
    g.set_boundaries(bc, bval)
    return g


def _run(L, g, st, fields, nsteps, launch=None):
    out = L.apply(g, st, fields, nsteps=nsteps, launch=launch)
    torch.cuda.synchronize()
    L.sync_status()
    return out if isinstance(out, list) else [out]


def _gs_fields(seed, shape):
    u = 1.0 - 0.3 * LI.uniform_field(seed, shape)
    v = 0.25 * LI.uniform_field(seed, shape, offset=int(np.prod(shape)))
    return [u, v]


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("bc", [[0, 0], [1, 0]])
def test_user_jacobi5_bitwise_equals_builtin(lope, dtype, bc):
    shape, T = (83, 264), 7
    u0 = to_device(LI.uniform_field(1200, shape), dtype)[0]
    g = _grid(lope, shape, dtype, 1, bc)
    user = lope.Stencil.source(JACOBI5, ndim=2, radius=1, params=[0.2])
    builtin = lope.Stencil.builtin("jacobi5", 0.2)
    for launch in (_launch(lope, TMA), _launch(lope, TRAP, 64, 32, 1), _launch(lope, TRAP, 32, 8, 3),
                   _launch(lope, DIRECT), _launch(lope, TMA, graph=1), None):
        a = _run(lope, g, user, u0, T, launch)[0]
        b = _run(lope, g, builtin, u0, T, launch)[0]
        assert torch.equal(a, b), launch
    for scheme in ("rk2", "rk3"):
        user.set_scheme(scheme)
        builtin.set_scheme(scheme)
        for launch in (_launch(lope, TMA), _launch(lope, TRAP, 64, 16, 1), _launch(lope, DIRECT)):
            a = _run(lope, g, user, u0, 3, launch)[0]
            b = _run(lope, g, builtin, u0, 3, launch)[0]
            assert torch.equal(a, b), (scheme, launch)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_user_diff7_bitwise_equals_builtin(lope, dtype):
    shape, T = (37, 50, 72), 6
    u0 = to_device(LI.uniform_field(1201, shape), dtype)[0]
    g = _grid(lope, shape, dtype, 1, [1, 0, 1])
    user = lope.Stencil.source(DIFF7, ndim=3, radius=1, params=[0.1])
    builtin = lope.Stencil.builtin("diff7", 0.1)
    for launch in (_launch(lope, TMA), _launch(lope, DIRECT)):
        assert torch.equal(_run(lope, g, user, u0, T, launch)[0],
                           _run(lope, g, builtin, u0, T, launch)[0]), launch


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_user_two_sweeps_per_launch_bitwise_equals_builtin(lope, dtype):
    """Two sweeps per launch (the planner's choice on large grids) run a
    user-written star function through the builtins' two-sweep kernels: the
    3D march with shared u1 planes (x and y sides Dirichlet 0, z periodic or
    not) and the 2D tiles (periodic and Dirichlet sides); bitwise equal to
    the builtin on the same launch and to one sweep per launch."""
    T = 7  # odd: the last launch runs one sweep
    k2, k1 = _launch(lope, TMA, k=2), _launch(lope, TMA, k=1)
    shape3 = (37, 50, 72)
    u3 = to_device(LI.uniform_field(1203, shape3), dtype)[0]
    user3 = lope.Stencil.source(DIFF7, ndim=3, radius=1, params=[0.1])
    builtin3 = lope.Stencil.builtin("diff7", 0.1)
    for bc in ([1, 1, 1], [0, 1, 1]):
        g = _grid(lope, shape3, dtype, 1, bc)
        a = _run(lope, g, user3, u3, T, k2)[0]
        assert torch.equal(a, _run(lope, g, builtin3, u3, T, k2)[0]), bc
        assert torch.equal(a, _run(lope, g, builtin3, u3, T, k1)[0]), bc
    shape2 = (83, 264)
    u2 = to_device(LI.uniform_field(1204, shape2), dtype)[0]
    user2 = lope.Stencil.source(JACOBI5, ndim=2, radius=1, params=[0.2])
    builtin2 = lope.Stencil.builtin("jacobi5", 0.2)
    for bc in ([0, 0], [1, 1], [1, 0]):
        g = _grid(lope, shape2, dtype, 1, bc)
        a = _run(lope, g, user2, u2, T, k2)[0]
        assert torch.equal(a, _run(lope, g, builtin2, u2, T, k2)[0]), bc
        assert torch.equal(a, _run(lope, g, builtin2, u2, T, k1)[0]), bc
    # two coupled fields (Gray-Scott, no builtin): both warp layouts of the
    # multi-field tiles against one sweep per launch
    gs = [to_device(x, dtype)[0] for x in _gs_fields(1205, shape2)]
    usr = lope.Stencil.source(GRAY_SCOTT, ndim=2, radius=1, nfields=2, params=GRAY_SCOTT_PRM)
    for bc in ([0, 0], [1, 0]):
        g = _grid(lope, shape2, dtype, 1, bc, nf=2)
        ref = _run(lope, g, usr, gs, T, k1)
        for ty in (0, 1):
            got = _run(lope, g, usr, gs, T, _launch(lope, TMA, 0, ty, 2))
            assert all(torch.equal(x, y) for x, y in zip(got, ref)), (bc, ty)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
def test_user_swe_flux_bitwise_equals_builtin(lope, dtype):
    shape, T = (83, 264), 5
    h, u, v = LI.swe_fields(1202, shape)
    dev = [to_device(x, dtype)[0] for x in (h - 1.0, u, v)]
    g = _grid(lope, shape, dtype, 1, [0, 0], nf=3)
    user = lope.Stencil.source(SWE_FLUX, ndim=2, radius=1, nfields=3, params=FLUX, box=True)
    builtin = lope.Stencil.builtin("swe_flux", *FLUX)
    launches = [_launch(lope, TMA), _launch(lope, TRAP, 64, 32, 1), _launch(lope, DIRECT)]
    if dtype != "f64":
        launches.append(_launch(lope, TMA, k=2))  # two sweeps per launch, box halo
    for launch in launches:
        a = _run(lope, g, user, dev, T, launch)
        b = _run(lope, g, builtin, dev, T, launch)
        for k in range(3):
            assert torch.equal(a[k], b[k]), (launch, k)


@pytest.mark.parametrize("scheme", ["euler", "rk3"])
@pytest.mark.parametrize("bc,bval", [([0, 0], None), ([1, 1], [(1.0, 1.0), (0.0, 0.0)])])
def test_gray_scott_fp64_vs_oracle_every_path(lope, orc, scheme, bc, bval):
    shape, T = (70, 136), 12
    fl = _gs_fields(1203, shape)
    dev, stored = zip(*(to_device(f, "f64") for f in fl))
    g = _grid(lope, shape, "f64", 1, bc, bval, nf=2)
    st = lope.Stencil.source(GRAY_SCOTT, ndim=2, radius=1, nfields=2, params=GRAY_SCOTT_PRM)
    st.set_scheme(scheme)
    want = orc.apply_source(list(stored), GRAY_SCOTT, GRAY_SCOTT_PRM, T, bc=bc, bval=bval,
                            scheme=scheme)
    paths = [None, _launch(lope, TRAP, 64, 16, 1), _launch(lope, DIRECT)]
    if bval is None:
        paths.append(_launch(lope, TMA))
    for launch in paths:
        outs = _run(lope, g, st, list(dev), T, launch)
        for k in range(2):
            assert normwise(to_host(outs[k]), want[k]) <= 1e-12, (launch, k)


def test_gray_scott_f32_bound_and_paths_bitwise(lope, orc, error_report):
    """FP32 Gray-Scott against the oracle within the elementwise first-order
    bound of error_bounds.py (local error from the body's operation tree,
    carried by |J_t| along the oracle's trajectory; below 1e-3 here)."""
    shape, T = (100, 200), 20
    fl = _gs_fields(1204, shape)
    dev, stored = zip(*(to_device(f, "f32") for f in fl))
    g = _grid(lope, shape, "f32", 1, [0, 0], nf=2)
    st = lope.Stencil.source(GRAY_SCOTT, ndim=2, radius=1, nfields=2, params=GRAY_SCOTT_PRM)
    B, want = gray_scott_majorant(orc, GRAY_SCOTT, GRAY_SCOTT_PRM, list(stored), T)
    assert max(float(np.max(b)) for b in B) < 1e-3
    ref = _run(lope, g, st, list(dev), T, _launch(lope, TMA))
    worst = []
    for k in range(2):
        err = np.abs(to_host(ref[k]) - want[k])
        worst.append(float(np.max(err)))
        assert np.all(err <= B[k]), (k, float(np.max(err / B[k])))
    error_report["F4 Gray-Scott source FP32 100x200 x20"] = {
        "max_abs": worst, "bound": [float(np.max(b)) for b in B]}
    for launch in (_launch(lope, TRAP, 64, 32, 2), _launch(lope, DIRECT)):
        outs = _run(lope, g, st, list(dev), T, launch)
        for k in range(2):
            assert torch.equal(outs[k], ref[k]), (launch, k)


def test_source_error_surfaces_at_launch(lope):
    g = _grid(lope, (32, 32), "f32", 1, [0, 0])
    st = lope.Stencil.source("out[0] = U(0, 0, 0) * no_such_thing;", params=[1.0])
    u0 = torch.zeros(32, 32, device="cuda")
    with pytest.raises(lope.LopeError, match="no_such_thing"):
        lope.apply(g, st, u0, nsteps=1)


def test_full_size_gray_scott_2048_sampled(lope, orc):
    """Gray-Scott at 2048^2 x 2 fields, FP32, periodic, 100 steps on the TMA
    tiles: sampled points against the oracle on their domain of dependence.
    Stated bound 1e-4 (100 steps of about 12 roundings of 2^-24 on values
    <= 1, with the per-step growth G of the test above bounded by 1.1)."""
    from gpu_helpers import sub_box

    shape, T = (2048, 2048), 100
    fl = _gs_fields(1205, shape)
    dev, stored = zip(*(to_device(f, "f32") for f in fl))
    g = _grid(lope, shape, "f32", 1, [0, 0], nf=2)
    st = lope.Stencil.source(GRAY_SCOTT, ndim=2, radius=1, nfields=2, params=GRAY_SCOTT_PRM)
    outs = _run(lope, g, st, list(dev), T)
    for p in [(0, 0), (2047, 2047), (1024, 5), (3, 1500)]:
        idx, pos = sub_box(shape, p, T + 1, [True, True])
        sub = [s[np.ix_(*idx)] for s in stored]
        want = orc.apply_source(sub, GRAY_SCOTT, GRAY_SCOTT_PRM, T, bc=[1, 1],
                                bval=[(1.0, 1.0), (0.0, 0.0)], nthreads=orc.max_threads())
        for k in range(2):
            assert abs(float(outs[k][p].item()) - want[k][pos]) <= 1e-4, (p, k)


GRAY_SCOTT_3D = """
const C u = U(0, 0, 0, 0), v = U(1, 0, 0, 0);
const C nu = add(add(add(U(0, -1, 0, 0), U(0, 1, 0, 0)), add(U(0, 0, -1, 0), U(0, 0, 1, 0))),
                 add(U(0, 0, 0, -1), U(0, 0, 0, 1)));
const C nv = add(add(add(U(1, -1, 0, 0), U(1, 1, 0, 0)), add(U(1, 0, -1, 0), U(1, 0, 1, 0))),
                 add(U(1, 0, 0, -1), U(1, 0, 0, 1)));
const C uvv = mul(u, mul(v, v));
out[0] = fma_(P[0], fma_(P[1], fma_(C(-6), u, nu), fma_(P[3], sub(C(1), u), -uvv)), u);
out[1] = fma_(P[0], fma_(P[2], fma_(C(-6), v, nv), fma_(-add(P[3], P[4]), v, uvv)), v);
"""

THREE_FIELD_3D = """
// three coupled fields, radius 2 along z (a 3D ring with three fields per stage)
for (int f = 0; f < 3; ++f) {
  const int g = (f + 1) % 3;
  out[f] = fma_(P[0], sub(add(U(g, 0, 0, -2), U(g, 0, 0, 2)), add(U(f, 1, 0, 0), U(f, 0, -1, 0))),
                U(f, 0, 0, 0));
}
"""

BOX_3D = """
out[0] = fma_(P[0], sub(add(U(0, 1, 1, 1), U(0, -1, -1, -1)), mul(C(2), U(0, 0, 0, 0))), U(0, 0, 0, 0));
"""


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_user_3d_two_and_three_fields_vs_oracle(lope, orc, dtype):
    shape, T = (21, 37, 72), 6
    for body, nf, prm, radius in ((GRAY_SCOTT_3D, 2, [0.5, 0.08, 0.04, 0.035, 0.065], 1),
                                  (THREE_FIELD_3D, 3, [0.05], 2)):
        fl = [LI.uniform_field(1400 + k, shape) for k in range(nf)]
        dev, stored = zip(*(to_device(f, dtype) for f in fl))
        g = _grid(lope, shape, dtype, radius, [0, 1, 0], nf=nf)
        st = lope.Stencil.source(body, ndim=3, radius=radius, nfields=nf, params=prm)
        want = orc.apply_source(list(stored), body, prm, T, bc=[0, 1, 0])
        ref = _run(lope, g, st, list(dev), T, _launch(lope, TMA))
        for launch in (_launch(lope, DIRECT), None):
            outs = _run(lope, g, st, list(dev), T, launch)
            for k in range(nf):
                assert torch.equal(outs[k], ref[k]), (nf, launch, k)
        for k in range(nf):
            got = to_host(ref[k])
            if dtype == "f64":
                assert normwise(got, want[k]) <= 1e-12, (nf, k)
            else:
                tol = 0.05 if dtype == "bf16" else 2e-5
                assert np.max(np.abs(got - want[k])) <= tol, (nf, k)


def test_user_3d_box_takes_direct_path(lope, orc):
    shape, T = (12, 20, 36), 4
    u0, u0s = to_device(LI.uniform_field(1410, shape), "f64")
    g = _grid(lope, shape, "f64", 1, [0, 0, 1])
    st = lope.Stencil.source(BOX_3D, ndim=3, radius=1, params=[0.1], box=True)
    with pytest.raises(lope.LopeError, match="does not support"):
        lope.apply(g, st, u0, nsteps=1, launch=_launch(lope, TMA))
    got = to_host(_run(lope, g, st, u0, T)[0])
    want = orc.apply_source(u0s, BOX_3D, [0.1], T, bc=[0, 0, 1])
    assert normwise(got, want) <= 1e-12


# 205 and 206 points per row: FP32 rows TMA cannot stage, starting at every
# 4-byte (205) or 8-byte (206) offset; 45 points: tiles narrower than the box.
@pytest.mark.parametrize("shape", [(12, 70, 205), (9, 67, 206), (21, 19, 45)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_user_3d_unaligned_rows_take_the_march(lope, orc, dtype, shape, capfd):
    """One-field star functions on rows TMA cannot stage run on the copied-plane
    z-march by default: bitwise the builtin diff7 on the march and the
    function's own direct kernel; a radius-2 function also matches the oracle
    (FP64: normwise 1e-12)."""
    T = 5
    u0, u0s = to_device(LI.uniform_field(1460, shape), dtype)
    bval = [(0.5, -0.3), -0.25, (1.0, 0.2)]
    for bc in ([1, 0, 1], [0, 0, 0], [1, 1, 1]):
        g = _grid(lope, shape, dtype, 1, bc, bval)
        user = lope.Stencil.source(DIFF7, ndim=3, radius=1, params=[0.1])
        lope.lope_set_option("log", 1)
        try:
            a = _run(lope, g, user, u0, T)[0]
        finally:
            lope.lope_set_option("log", 0)
        log = capfd.readouterr().err
        if (shape[2] * (8 if dtype == "f64" else 4)) % 16:  # rows TMA cannot stage
            assert "path=march" in log, bc
        builtin = lope.Stencil.builtin("diff7", 0.1)
        assert torch.equal(a, _run(lope, g, builtin, u0, T, _launch(lope, MARCH))[0]), bc
        assert torch.equal(a, _run(lope, g, user, u0, T, _launch(lope, DIRECT))[0]), bc
    bc = [1, 0, 0]
    g = _grid(lope, shape, dtype, 2, bc, bval)
    st = lope.Stencil.source(STAR_R2_3D, ndim=3, radius=2, params=[0.03, 0.05])
    a = _run(lope, g, st, u0, T, _launch(lope, MARCH))[0]
    assert torch.equal(a, _run(lope, g, st, u0, T, _launch(lope, DIRECT))[0])
    if dtype == "f64":
        want = orc.apply_source(u0s, STAR_R2_3D, [0.03, 0.05], T, bc=bc, bval=bval)
        assert normwise(to_host(a), want) <= 1e-12


def test_user_trapezoid_with_large_shared_memory(lope, orc):
    """Trapezoid tiles whose window needs more than 48 KB of shared memory
    (two fields, RK3, depth 2) after a smaller launch of the same function."""
    shape, T = (96, 200), 4
    fl = _gs_fields(1420, shape)
    dev, stored = zip(*(to_device(f, "f32") for f in fl))
    g = _grid(lope, shape, "f32", 1, [0, 0], nf=2)
    st = lope.Stencil.source(GRAY_SCOTT, ndim=2, radius=1, nfields=2, params=GRAY_SCOTT_PRM)
    st.set_scheme("rk3")
    small = _run(lope, g, st, list(dev), T, _launch(lope, TRAP, 64, 16, 1))
    for launch in (_launch(lope, TRAP, 64, 32, 2), _launch(lope, TRAP, 128, 32, 2)):
        outs = _run(lope, g, st, list(dev), T, launch)
        for k in range(2):
            assert torch.equal(outs[k], small[k]), (launch, k)


def test_computed_tap_outside_the_halo_is_reported_and_clamped(lope):
    """A tap whose offset is computed is checked when it runs: reading beyond
    the declared halo (Sec. 3.5) is clamped into it and lope_sync_status
    reports LOPE_ERR_INVALID; the context stays usable."""
    body = "C s = C(0);\nfor (int d = -2; d <= 2; d += 4) s = add(s, U(0, d, 0));\nout[0] = s;"
    st = lope.Stencil.source(body, ndim=2, radius=1)
    g = _grid(lope, (64, 128), "f32", 1, [0, 0])
    u = torch.rand(64, 128, device="cuda")
    for launch in (_launch(lope, TMA), _launch(lope, DIRECT)):
        lope.apply(g, st, u, nsteps=1, launch=launch)
        with pytest.raises(lope.LopeError, match="outside its declared halo"):
            lope.sync_status()
    ok = lope.Stencil.source("out[0] = add(U(0, -1, 0), U(0, 1, 0));", ndim=2, radius=1)
    out = lope.apply(g, ok, u, nsteps=1)
    lope.sync_status()
    assert torch.equal(out, torch.roll(u, 1, 1) + torch.roll(u, -1, 1))
