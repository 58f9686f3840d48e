"""GPU parity of box-halo local functions (corner taps) through the C ABI.

The nonlinear flux-form shallow water function "swe_flux" (three fields, a
radius-1 box halo, products of halo values) and linear box tables with corners
run on the 2D TMA tiles (wide box plus a per-warp halo-ring fill on wrapped
tiles), the trapezoid tiles and the direct kernel.  They are compared with the
FP64 oracle (FP64: normwise 1e-12; FP32/BF16: the bounds of gpu_helpers with
the step's infinity-norm growth G) and with each other bitwise.
"""
import numpy as np
import pytest
import torch

import lope_inputs as LI
from gpu_helpers import bound_bf16, bound_f32, normwise, to_device, to_host

pytestmark = pytest.mark.gpu

TMA, TRAP, DIRECT = 1, 2, 3
PRM = [0.02, 1.0, 0.5, 1.0]  # dt, g, f, H


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


def flux_fields(seed, shape):
    """(eta, u, v) = (0.01 N, 0.1 N, 0.1 N): h = 1 + 0.01 N stored as eta = h - H."""
    h, u, v = LI.swe_fields(seed, shape)
    return [h - 1.0, u, v]


def flux_growth(dt, g, f, H, Me, Mu):
    """Infinity-norm bound of one swe_flux step's Jacobian for |eta| <= Me and
    |u|, |v| <= Mu (row sums of the absolute partial derivatives)."""
    mass = 1 + dt * (4 * (H + Me) + 4 * Mu)
    mom = 1 + dt * (abs(f) + 2 * g + 4 * Mu + 2 * Mu)
    return max(mass, mom)


BCS = [([0, 0], None), ([1, 0], None), ([0, 1], None), ([1, 1], None)]


@pytest.mark.parametrize("bc,bval", BCS)
@pytest.mark.parametrize("path", [0, TMA, TRAP, DIRECT])
def test_swe_flux_fp64_1e12(lope, orc, bc, bval, path):
    shape, T = (70, 136), 15
    fields = flux_fields(1005, shape)
    dev, stored = zip(*(to_device(f, "f64") for f in fields))
    g = _grid(lope, shape, "f64", 1, bc, bval, nf=3)
    st = lope.Stencil.builtin("swe_flux", *PRM)
    launch = None if path == 0 else _launch(lope, path, 64, 16, 3 if path == TRAP else 1)
    outs = _run(lope, g, st, list(dev), T, launch)
    want = orc.apply(list(stored), "swe_flux", PRM, T, bc=bc, bval=bval)
    for k in range(3):
        assert normwise(to_host(outs[k]), want[k]) <= 1e-12, (k, bc, path)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_swe_flux_f32_bf16_vs_oracle(lope, orc, dtype):
    shape, T = (100, 200), 20
    fields = flux_fields(1006, shape)
    dev, stored = zip(*(to_device(f, dtype) for f in fields))
    st = lope.Stencil.builtin("swe_flux", *PRM)
    for bc in ([0, 0], [1, 0]):
        g = _grid(lope, shape, dtype, 1, bc, nf=3)
        want = orc.apply(list(stored), "swe_flux", PRM, T, bc=bc)
        Me = max(np.max(np.abs(stored[0])), np.max(np.abs(want[0])))
        Mu = max(np.max(np.abs(s)) for s in stored[1:] + tuple(want[1:]))
        G = flux_growth(*PRM, Me, Mu)
        M = max(Me, Mu)
        bound = bound_f32(T, M, 24, G) if dtype == "f32" else bound_bf16(T, M, 24, G)
        for launch in (None, _launch(lope, TRAP, 64, 32, 2), _launch(lope, DIRECT)):
            outs = _run(lope, g, st, list(dev), T, launch)
            for k in range(3):
                err = np.max(np.abs(to_host(outs[k]) - want[k]))
                assert err <= bound, (dtype, bc, k, launch, err, bound)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("bc", [[0, 0], [1, 1], [0, 1], [1, 0]])
def test_swe_flux_paths_bitwise(lope, dtype, bc):
    # 3 x 5 TMA tiles in f32 (64 x 32), ragged in both axes
    shape, T = (83, 264), 9
    dev = [to_device(f, dtype)[0] for f in flux_fields(1007, shape)]
    g = _grid(lope, shape, dtype, 1, bc, nf=3)
    st = lope.Stencil.builtin("swe_flux", *PRM)
    ref = _run(lope, g, st, dev, T, _launch(lope, TMA))
    for launch in (_launch(lope, DIRECT), _launch(lope, TRAP, 64, 32, 1),
                   _launch(lope, TRAP, 32, 8, 3), _launch(lope, TMA, graph=1)):
        outs = _run(lope, g, st, dev, T, launch)
        for k in range(3):
            assert torch.equal(outs[k], ref[k]), (launch, k)


def test_swe_flux_conserves_mass_on_gpu(lope):
    shape = (256, 320)
    dev = [to_device(f, "f64")[0] for f in flux_fields(1008, shape)]
    g = _grid(lope, shape, "f64", 1, [0, 0], nf=3)
    st = lope.Stencil.builtin("swe_flux", *PRM)
    outs = _run(lope, g, st, dev, 40)
    a = float(lope.reduce_sum(dev[0]).item())
    b = float(lope.reduce_sum(outs[0]).item())
    scale = float(lope.reduce_sum(dev[0].abs()).item())
    assert abs(a - b) <= 1e-13 * scale


def test_swe_flux_rejected_by_adjoint_and_bad_params(lope):
    g = _grid(lope, (32, 32), "f32", 1, [0, 0], nf=3)
    st = lope.Stencil.builtin("swe_flux", *PRM)
    with pytest.raises(lope.LopeError, match="single-field linear"):
        lope.workspace_size(g, st, 10, 5)
    with pytest.raises(lope.LopeError, match="parameter count"):
        lope.Stencil.builtin("swe_flux", 0.02, 1.0)


@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("bc", [[0, 0], [1, 0], [0, 1]])
def test_box_linear_tma_fp64_and_bitwise(lope, orc, r, bc):
    rng = np.random.default_rng(20 + r)
    w = rng.normal(size=(2 * r + 1, 2 * r + 1)) * 0.08
    w[r, r] = 0.4
    shape, T = (45, 100), 6
    u0, u0s = to_device(LI.uniform_field(30 + r, shape), "f64")
    g = _grid(lope, shape, "f64", r, bc)
    st = lope.Stencil.linear(w)
    want = orc.apply(u0s, "linear", nsteps=T, bc=bc, weights_table=w)
    ref = _run(lope, g, st, u0, T, _launch(lope, TMA))
    assert normwise(to_host(ref), want) <= 1e-12
    for launch in (_launch(lope, DIRECT), _launch(lope, TRAP, 32, 8, 2)):
        assert torch.equal(_run(lope, g, st, u0, T, launch), ref), launch
    # FP32 on the paired-column TMA tiles
    v0, v0s = to_device(LI.uniform_field(40 + r, shape), "f32")
    g32 = _grid(lope, shape, "f32", r, bc)
    ref32 = _run(lope, g32, st, v0, T, _launch(lope, TMA))
    want32 = orc.apply(v0s, "linear", nsteps=T, bc=bc, weights_table=w)
    G = float(np.abs(w).sum())
    assert np.max(np.abs(to_host(ref32) - want32)) <= bound_f32(T, 1.0, (2 * r + 1) ** 2 + 1, G)
    assert torch.equal(_run(lope, g32, st, v0, T, _launch(lope, DIRECT)), ref32)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_full_size_swe_flux_4096_200_sampled(lope, orc, dtype, error_report):
    """Nonlinear shallow water at 4096^2 x 3 fields, 200 steps, periodic.
    Sampled points are checked against the oracle on their domain of
    dependence.  FP32: the stated bound 2e-4 (linearised growth <= 1.4 over 200
    steps, about 24 roundings of 2^-24 per step on values <= 0.5); BF16: the
    storage-rounding bound with the same growth."""
    from test_gpu_parity import _sampled_check

    shape, T = (4096, 4096), 200
    fields = flux_fields(1009, shape)
    dev, stored = zip(*(to_device(f, dtype) for f in fields))
    g = _grid(lope, shape, dtype, 1, [0, 0], nf=3)
    st = lope.Stencil.builtin("swe_flux", *PRM)
    outs = _run(lope, g, st, list(dev), T)
    M = max(np.max(np.abs(s)) for s in stored)
    tol = (lambda k, w: 2e-4) if dtype == "f32" else (lambda k, w: 1.4 * T * (2.0 ** -9) * M)
    pts = [(0, 0), (4095, 4095), (2048, 17), (9, 3000)]
    worst = _sampled_check(lope, orc, "swe_flux", PRM, shape, [0, 0], T, 1, dtype, 3, outs,
                           list(stored), pts, tol)
    error_report[f"F1 swe_flux {dtype.upper()} 4096^2 x200 (sampled)"] = {
        "max_abs": worst, "bound": tol(0, 0.0)}
