"""GPU parity of the multi-stage (SSP Runge-Kutta) schemes through the C ABI.

A scheme's step is a sequence of sweeps of the local function with pointwise
combinations (see lope_stencil_set_scheme).  The trapezoid path fuses whole
steps in shared memory; the TMA and direct paths run one launch per stage with
the stage states in the work buffers.  Every path is compared with the FP64
oracle (FP64: normwise 1e-12) and with the others bitwise (each stage rounds to
the storage precision on every path, with the same operations in the same
order).
"""
import numpy as np
import pytest
import torch

import lope_inputs as LI
from gpu_helpers import bound_f32, normwise, to_device, to_host

pytestmark = pytest.mark.gpu

TMA, TRAP, DIRECT = 1, 2, 3
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
    return out


def _fields(kind, shape, seed):
    if kind == "swe_flux":
        h, u, v = LI.swe_fields(seed, shape)
        return [h - 1.0, u, v]
    return [LI.uniform_field(seed, shape)]


CASES = [  # kind, params, halo, shape, bc, bval
    ("jacobi5", [0.2], 1, (70, 136), [0, 0], None),
    ("jacobi5", [0.2], 1, (70, 136), [1, 1], [0.25, -0.5]),
    ("star9r2", [0.1], 2, (45, 72), [0, 1], None),
    ("swe_flux", FLUX, 1, (50, 136), [0, 0], None),
    ("swe_flux", FLUX, 1, (50, 136), [1, 0], None),
    ("diff7", [0.1], 1, (20, 24, 40), [1, 1, 1], None),
    ("diff7", [0.1], 1, (20, 24, 40), [0, 1, 0], None),
]


@pytest.mark.parametrize("scheme", ["rk2", "rk3"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[4]}")
def test_rk_fp64_all_paths_vs_oracle(lope, orc, scheme, case):
    kind, prm, halo, shape, bc, bval = case
    T = 6
    fl = _fields(kind, shape, 1100)
    dev, stored = zip(*(to_device(f, "f64") for f in fl))
    g = _grid(lope, shape, "f64", halo, bc, bval, nf=len(fl))
    st = lope.Stencil.builtin(kind, *prm).set_scheme(scheme)
    want = orc.apply(list(stored) if len(fl) > 1 else stored[0], kind, prm, T, bc=bc, bval=bval,
                     scheme=scheme)
    want = want if len(fl) > 1 else [want]
    paths = [None, _launch(lope, DIRECT)]
    if len(shape) == 2:
        paths += [_launch(lope, TRAP, 64, 16, 1), _launch(lope, TRAP, 32, 8, 2)]
    if bval is None:  # the TMA tiles take Dirichlet-0 halos only
        paths.append(_launch(lope, TMA))
    for launch in paths:
        outs = _run(lope, g, st, list(dev), T, launch)
        outs = outs if isinstance(outs, list) else [outs]
        for k in range(len(fl)):
            assert normwise(to_host(outs[k]), want[k]) <= 1e-12, (launch, k)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("scheme", ["rk2", "rk3"])
@pytest.mark.parametrize("kind,prm,halo", [("jacobi5", [0.2], 1), ("star9r2", [0.1], 2),
                                           ("swe_flux", FLUX, 1)])
def test_rk_2d_paths_bitwise(lope, dtype, scheme, kind, prm, halo):
    shape, T = (83, 264), 5
    fl = [to_device(f, dtype)[0] for f in _fields(kind, shape, 1101)]
    for bc in ([0, 0], [1, 0]):
        g = _grid(lope, shape, dtype, halo, bc, nf=len(fl))
        st = lope.Stencil.builtin(kind, *prm).set_scheme(scheme)
        ref = _run(lope, g, st, fl, T, _launch(lope, TMA))
        ref = ref if isinstance(ref, list) else [ref]
        for launch in (_launch(lope, DIRECT), _launch(lope, TRAP, 64, 32, 1),
                       _launch(lope, TRAP, 32, 16, 3), None):
            outs = _run(lope, g, st, fl, T, launch)
            outs = outs if isinstance(outs, list) else [outs]
            for k in range(len(fl)):
                assert torch.equal(outs[k], ref[k]), (bc, launch, k)


@pytest.mark.parametrize("scheme", ["rk2", "rk3"])
def test_rk_3d_tma_direct_bitwise_and_bound(lope, orc, scheme):
    shape, c, T = (37, 50, 72), 0.1, 5
    u0, u0s = to_device(LI.uniform_field(1102, shape), "f32")
    g = _grid(lope, shape, "f32", 1, [1, 0, 1])
    st = lope.Stencil.builtin("diff7", c).set_scheme(scheme)
    ref = _run(lope, g, st, u0, T, _launch(lope, TMA))
    assert torch.equal(_run(lope, g, st, u0, T, _launch(lope, DIRECT)), ref)
    want = orc.apply(u0s, "diff7", [c], T, bc=[1, 0, 1], scheme=scheme)
    stages = 2 if scheme == "rk2" else 3
    # each stage: the 9 roundings of one sweep plus 2 of the combination; the
    # step is a convex combination of Euler steps (non-expansive in max norm)
    assert np.max(np.abs(to_host(ref) - want)) <= bound_f32(T, 1.0, stages * 11)


def test_rk_work_states_and_rejections(lope):
    st = lope.Stencil.builtin("jacobi5", 0.2)
    assert st.work_states() == 1
    assert st.set_scheme("rk2").work_states() == 1
    assert st.set_scheme("rk3").work_states() == 2
    shape = (64, 64)
    g = _grid(lope, shape, "f32", 1, [0, 0])
    u0, _ = to_device(LI.uniform_field(1103, shape), "f32")
    out = torch.empty_like(u0)
    # RK3 on the stage path needs two work states; a one-state buffer that sits
    # right before `out` overlaps it
    buf = torch.empty((2,) + shape, device="cuda")
    with pytest.raises(lope.LopeError, match="alias"):
        lope.apply(g, st, u0, out=buf[1], work=buf[0], nsteps=1, launch=_launch(lope, TMA))
    with pytest.raises(lope.LopeError, match="multi-stage"):
        lope.workspace_size(g, st, 10, 5)
    with pytest.raises(lope.LopeError, match="forward-Euler"):
        lope.apply_batch([g], st, [u0], nsteps=2)
    with pytest.raises(lope.LopeError):
        lope.lope_stencil_set_scheme(st.handle, 4)
    # nsteps = 1 and 0 with a multi-stage scheme
    w = torch.empty((2,) + shape, device="cuda")
    lope.apply(g, st, u0, out=out, work=w, nsteps=0)
    torch.cuda.synchronize()
    assert torch.equal(out, u0)


def test_rk3_mass_conserved_swe_flux_on_gpu(lope):
    shape = (128, 192)
    fl = [to_device(f, "f64")[0] for f in _fields("swe_flux", shape, 1104)]
    g = _grid(lope, shape, "f64", 1, [0, 0], nf=3)
    st = lope.Stencil.builtin("swe_flux", *FLUX).set_scheme("rk3")
    outs = _run(lope, g, st, fl, 20)
    a = float(lope.reduce_sum(fl[0]).item())
    b = float(lope.reduce_sum(outs[0]).item())
    assert abs(a - b) <= 1e-13 * float(lope.reduce_sum(fl[0].abs()).item())


def test_full_size_rk3_swe_flux_4096_sampled(lope, orc, error_report):
    """RK3 steps of the nonlinear shallow water at 4096^2, periodic, 50 steps
    (150 sweeps): sampled points against the oracle on their domain of
    dependence (R * stages * T cells).  Stated FP32 bound 1e-4 (150 sweeps of
    about 26 roundings on values <= 0.5, linearised growth <= 1.2)."""
    from test_gpu_parity import sub_box

    shape, T = (4096, 4096), 50
    fl = _fields("swe_flux", shape, 1105)
    dev, stored = zip(*(to_device(f, "f32") for f in fl))
    g = _grid(lope, shape, "f32", 1, [0, 0], nf=3)
    st = lope.Stencil.builtin("swe_flux", *FLUX).set_scheme("rk3")
    outs = _run(lope, g, st, list(dev), T)
    rho = 3 * T + 1
    worst = [0.0] * 3
    for p in [(0, 0), (4095, 4095), (2048, 17), (9, 3000)]:
        idx, pos = sub_box(shape, p, rho, [True, True])
        sub = [s[np.ix_(*idx)] for s in stored]
        want = orc.apply(sub, "swe_flux", FLUX, T, bc=[1, 1], scheme="rk3",
                         nthreads=orc.max_threads())
        for k in range(3):
            err = abs(float(outs[k][p].item()) - want[k][pos])
            worst[k] = max(worst[k], err)
            assert err <= 1e-4, (p, k)
    error_report["F2 RK3 swe_flux FP32 4096^2 x50 (sampled)"] = {"max_abs": worst, "bound": 1e-4}


@pytest.mark.parametrize("scheme", ["rk2", "rk3"])
def test_rk_bf16_vs_oracle_and_single_step(lope, orc, scheme):
    shape = (64, 200)
    u0, u0s = to_device(LI.uniform_field(1106, shape), "bf16")
    g = _grid(lope, shape, "bf16", 1, [1, 0])
    st = lope.Stencil.builtin("jacobi5", 0.2).set_scheme(scheme)
    for T in (1, 7):
        want = orc.apply(u0s, "jacobi5", [0.2], T, bc=[1, 0], scheme=scheme)
        stages = 2 if scheme == "rk2" else 3
        # every stage rounds to BF16 (2^-9 relative), the step is non-expansive
        bound = T * stages * (2.0 ** -9 + 11 * 2.0 ** -24) * 1.0001
        for launch in (None, _launch(lope, TMA), _launch(lope, DIRECT)):
            got = to_host(_run(lope, g, st, u0, T, launch))
            assert got.shape == want.shape
            assert np.max(np.abs(got - want)) <= bound, (T, launch)
