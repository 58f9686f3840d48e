"""External halos and slab decomposition on the GPU.

A grid with LOPE_BC_EXTERNAL sides reads the halo of its slowest axis from
the caller's buffer beyond the grid (the planes a halo exchange delivers).  A
slab swept that way must equal the same planes of the whole-grid sweep
bitwise, on the TMA path (2D tiles, 3D z-march) and the direct kernel.  The
slab runner (paper_1502_03504_gb300.slab) then advances a grid cut into 2 or
3 slabs on one device, exchanging ghost planes by device-to-device copies on a
second stream, border planes first, and must equal the whole-grid run bitwise
(and the FP64 oracle within its bound).
"""
import numpy as np
import pytest
import torch

import lope_inputs as LI
from gpu_helpers import to_device, to_host
from paper_1502_03504_gb300.slab import (BC_DIRICHLET, BC_EXTERNAL, BC_PERIODIC, LocalTransport,
                                         LopeSweeper, SlabPlan, SlabRunner)

pytestmark = pytest.mark.gpu

TMA, DIRECT = 1, 3
TORCH = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}


def _whole(lope, shape, dtype, halo, slow, other, nf):
    g = lope.Grid(shape, dtype, halo=halo, nfields=nf)
    (klo, vlo), (khi, vhi) = slow
    bcs, vals = [(klo, khi) if klo != BC_PERIODIC else 0], [(vlo, vhi)]
    for b in other:
        bcs.append(b)
        vals.append(0.0)
    g.set_boundaries(bcs, vals)
    return g


@pytest.mark.parametrize("path", [TMA, DIRECT])
@pytest.mark.parametrize("case", [
    ("diff7", [0.1], (24, 40, 72), "f32", 1, [1, 1]),
    ("diff7", [0.1], (24, 40, 72), "f32", 1, [0, 0]),
    ("star9r2", [0.1], (90, 136), "f32", 2, [0]),
    ("swe_flux", [0.02, 1.0, 0.5, 1.0], (70, 64), "f32", 1, [0]),
    ("jacobi5", [0.2], (50, 70), "f64", 1, [1]),
], ids=lambda c: f"{c[0]}-{c[3]}-{'x'.join(map(str, c[2]))}-{c[5]}")
def test_external_halo_sweep_equals_whole_grid_planes(lope, path, case):
    kind, prm, shape, dtype, R, other = case
    nf = 3 if kind.startswith("swe") else 1
    fields = [to_device(LI.uniform_field(2100 + f, shape) * (0.1 if nf > 1 else 1.0), dtype)[0]
              for f in range(nf)]
    st = lope.Stencil.builtin(kind, *prm)
    whole = _whole(lope, shape, dtype, R, ((BC_PERIODIC, 0.0), (BC_PERIODIC, 0.0)), other, nf)
    ref = lope.apply(whole, st, fields if nf > 1 else fields[0], nsteps=1,
                     launch=lope.Launch(path, 0, 0, 0, -1))
    ref = ref if nf > 1 else [ref]
    a, b = 7, shape[0] - 9  # the slab: planes [a, b), R ghost planes beyond each side
    slab = lope.Grid((b - a,) + shape[1:], dtype, halo=R, nfields=nf)
    slab.set_boundaries([(BC_EXTERNAL, BC_EXTERNAL)] + other)
    ext = [x[a - R:b + R].clone() for x in fields]  # the caller's buffer, ghosts included
    ins = [e[R:R + b - a] for e in ext]
    outs = [torch.full_like(i, float("nan")) for i in ins]
    lope.apply(slab, st, ins if nf > 1 else ins[0], out=outs if nf > 1 else outs[0], nsteps=1,
               launch=lope.Launch(path, 0, 0, 0, -1))
    torch.cuda.synchronize()
    lope.sync_status()
    for f in range(nf):
        assert torch.equal(outs[f], ref[f][a:b]), f
    # one external side, the grid's own boundary on the other
    lo = lope.Grid((b,) + shape[1:], dtype, halo=R, nfields=nf)
    lo.set_boundaries([(BC_DIRICHLET, BC_EXTERNAL)] + other)
    whole_d = _whole(lope, shape, dtype, R, ((BC_DIRICHLET, 0.0), (BC_DIRICHLET, 0.0)), other, nf)
    ref_d = lope.apply(whole_d, st, fields if nf > 1 else fields[0], nsteps=1,
                       launch=lope.Launch(path, 0, 0, 0, -1))
    ref_d = ref_d if nf > 1 else [ref_d]
    buf = [x[:b + R].clone() for x in fields]
    ins = [x[:b] for x in buf]
    outs = [torch.full_like(i, float("nan")) for i in ins]
    lope.apply(lo, st, ins if nf > 1 else ins[0], out=outs if nf > 1 else outs[0], nsteps=1,
               launch=lope.Launch(path, 0, 0, 0, -1))
    torch.cuda.synchronize()
    for f in range(nf):
        assert torch.equal(outs[f], ref_d[f][:b]), f


def test_external_halo_refusals(lope):
    shape = (32, 64)
    g = lope.Grid(shape, "f32", halo=1)
    g.set_boundaries([(BC_EXTERNAL, BC_EXTERNAL), 0])
    st = lope.Stencil.builtin("jacobi5", 0.2)
    buf = torch.zeros((34, 64), device="cuda")
    u = buf[1:33]
    with pytest.raises(lope.LopeError, match="one sweep per call"):
        lope.apply(g, st, u, nsteps=3)
    with pytest.raises(lope.LopeError, match="UNSUPPORTED"):
        lope.apply(g, st, u, nsteps=1, launch=lope.Launch(2, 64, 16, 1, -1))
    with pytest.raises(lope.LopeError, match="aliases"):  # out inside in's halo planes
        lope.apply(g, st, u, out=buf[2:34], nsteps=1)


def _runner(lope, kind, prm, shape, dtype, R, k, parts, slow, other):
    nf = 3 if kind.startswith("swe") else 1
    plan = SlabPlan(shape[0], parts, R, k, *slow)
    st = lope.Stencil.builtin(kind, *prm)
    bnd = [((b, 0.0), (b, 0.0)) for b in other]
    sweep = LopeSweeper(lope, st, shape, dtype, R, nf, bnd)

    def alloc(planes, slab):
        return [torch.full((planes,) + tuple(shape[1:]), float("nan"), dtype=TORCH[dtype],
                           device="cuda") for _ in range(nf)]

    streams = (torch.cuda.current_stream(), torch.cuda.Stream())
    return SlabRunner(plan, range(parts), sweep, LocalTransport(), alloc, streams), st, nf


@pytest.mark.parametrize("case", [
    ("diff7", [0.1], (60, 40, 72), "f32", 1, ((BC_DIRICHLET, 0.0), (BC_DIRICHLET, 0.0)), [1, 1], 2),
    ("diff7", [0.1], (61, 33, 64), "f32", 1, ((BC_PERIODIC, 0.0), (BC_PERIODIC, 0.0)), [1, 0], 3),
    ("star9r2", [0.1], (200, 136), "f32", 2, ((BC_PERIODIC, 0.0), (BC_PERIODIC, 0.0)), [0], 2),
    ("swe_flux", [0.02, 1.0, 0.5, 1.0], (130, 136), "f32", 1,
     ((BC_PERIODIC, 0.0), (BC_PERIODIC, 0.0)), [0], 3),
    ("jacobi5", [0.2], (90, 64), "f32", 1, ((BC_DIRICHLET, 0.3), (BC_DIRICHLET, -0.2)), [0], 2),
], ids=lambda c: f"{c[0]}-{'x'.join(map(str, c[2]))}-{c[7]}slabs")
@pytest.mark.parametrize("k", [1, 3])
def test_slab_runner_equals_whole_grid(lope, orc, case, k):
    kind, prm, shape, dtype, R, slow, other, parts = case
    T = 7
    runner, st, nf = _runner(lope, kind, prm, shape, dtype, R, k, parts, slow, other)
    fields64 = [LI.uniform_field(2200 + f, shape) * (0.1 if nf > 1 else 1.0) for f in range(nf)]
    dev, stored = zip(*(to_device(f, dtype) for f in fields64))
    runner.scatter(list(dev))
    runner.run(T)
    got = [torch.full_like(x, float("nan")) for x in dev]
    runner.gather(got)
    torch.cuda.synchronize()
    lope.sync_status()
    whole = _whole(lope, shape, dtype, R, slow, other, nf)
    ref = lope.apply(whole, st, list(dev) if nf > 1 else dev[0], nsteps=T)
    ref = ref if nf > 1 else [ref]
    torch.cuda.synchronize()
    for f in range(nf):
        assert torch.equal(got[f], ref[f]), f
    if k == 3 and kind == "diff7":
        (klo, vlo), (khi, vhi) = slow
        want = orc.apply(stored[0], kind, prm, T,
                         bc=[(klo, khi) if klo != BC_PERIODIC else 0] + other,
                         bval=[(vlo, vhi)] + [0.0] * len(other))
        assert np.max(np.abs(to_host(got[0]) - want)) <= T * 5 * 2.0 ** -24
