"""The two-sweep 3D z-march (TMA path, temporal depth 2).

One launch applies the local function twice, keeping the intermediate state
on chip; every sweep rounds to the storage precision, so the result must equal
one sweep per launch bitwise (and the direct kernel), on grids with ragged
tiles in every axis, Dirichlet-0 x and y sides, Dirichlet or periodic z, both
tile heights, FP32 and BF16 storage, even and odd step counts (an odd count
ends with a one-sweep launch).  One case per shape is checked against the FP64
oracle within the derived bound, and the kernel writes only its output.
"""
import numpy as np
import pytest
import torch

import lope_inputs as LI
from error_bounds import local_eps
from gpu_helpers import to_device, to_host

pytestmark = pytest.mark.gpu

TMA, DIRECT = 1, 3
SHORT, TALL = 1, 2


def _run(L, g, st, u, T, launch, out=None, work=None):
    o = L.apply(g, st, u, out=out, work=work, nsteps=T, launch=launch)
    torch.cuda.synchronize()
    L.sync_status()
    return o


def _grid(L, shape, dtype, zbc):
    g = L.Grid(shape, dtype, halo=1)
    g.set_boundaries([zbc, 1, 1])
    return g


SHAPES = [(37, 50, 72), (40, 130, 136), (5, 64, 64), (70, 33, 200), (1, 8, 8)]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("zbc", [1, 0])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_two_sweeps_bitwise_equal_one_sweep(lope, orc, dtype, zbc, shape):
    u0, u0s = to_device(LI.uniform_field(1700, shape), dtype)
    g = _grid(lope, shape, dtype, zbc)
    st = lope.Stencil.builtin("diff7", 0.1)
    for T in (2, 7):
        ref = _run(lope, g, st, u0, T, lope.Launch(TMA, 0, 0, 1, -1))
        direct = _run(lope, g, st, u0, T, lope.Launch(DIRECT, 0, 0, 0, -1))
        assert torch.equal(ref, direct)
        for tx, ty in ((0, SHORT), (0, TALL), (1, 0)):  # per-warp slots; block-shared planes
            got = _run(lope, g, st, u0, T, lope.Launch(TMA, tx, ty, 2, -1))
            assert torch.equal(got, ref), (T, tx, ty)
        if dtype == "f32" and T == 7:
            want = orc.apply(u0s, "diff7", [0.1], T, bc=[zbc, 1, 1])
            bound = T * float(local_eps("diff7", [0.1], [float(np.max(np.abs(u0s)))], "f32")[0])
            assert np.max(np.abs(to_host(ref) - want)) <= bound


def test_two_sweeps_linear_table_asymmetric(lope):
    """An asymmetric radius-1 star table: any transposed tap shows up."""
    w = np.zeros((3, 3, 3))
    rng = np.random.default_rng(1701)
    for ax in range(3):
        for d in (0, 2):
            idx = [1, 1, 1]
            idx[ax] = d
            w[tuple(idx)] = rng.uniform(0.02, 0.12)
    w[1, 1, 1] = 1.0 - w.sum()
    shape = (33, 70, 136)
    u0, _ = to_device(LI.uniform_field(1702, shape), "f32")
    st = lope.Stencil.linear(w)
    for zbc in (0, 1):
        g = _grid(lope, shape, "f32", zbc)
        ref = _run(lope, g, st, u0, 6, lope.Launch(DIRECT, 0, 0, 0, -1))
        for tx, ty in ((0, SHORT), (0, TALL), (1, 0)):
            assert torch.equal(_run(lope, g, st, u0, 6, lope.Launch(TMA, tx, ty, 2, -1)), ref)


def test_two_sweeps_refused_where_it_does_not_apply(lope):
    shape = (16, 32, 64)
    u0 = torch.rand(shape, device="cuda")
    st = lope.Stencil.builtin("diff7", 0.1)
    g = lope.Grid(shape, "f32", halo=1)  # periodic x and y: the one-sweep march only
    with pytest.raises(lope.LopeError, match="UNSUPPORTED"):
        lope.apply(g, st, u0, nsteps=4, launch=lope.Launch(TMA, 0, 0, 2, -1))
    g.set_boundaries([1, 1, 1], [0.0, 0.5, 0.0])  # non-zero Dirichlet value
    with pytest.raises(lope.LopeError, match="UNSUPPORTED"):
        lope.apply(g, st, u0, nsteps=4, launch=lope.Launch(TMA, 0, 0, 2, -1))


def test_two_sweeps_write_only_their_output(lope):
    shape = (21, 70, 136)
    n = int(np.prod(shape))
    guard, sentinel = 4096, -7.0e30
    u0, _ = to_device(LI.uniform_field(1703, shape), "f32")
    keep = u0.clone()
    g = _grid(lope, shape, "f32", 1)
    st = lope.Stencil.builtin("diff7", 0.1)
    bufs = [torch.full((n + 2 * guard,), sentinel, device="cuda") for _ in range(2)]
    out, work = (b[guard:guard + n].view(shape) for b in bufs)
    for tx, ty in ((0, SHORT), (0, TALL), (1, 0)):
        _run(lope, g, st, u0, 5, lope.Launch(TMA, tx, ty, 2, -1), out=out, work=work)
        for b in bufs:
            assert bool((b[:guard] == sentinel).all()) and bool((b[guard + n:] == sentinel).all())
        assert torch.equal(u0, keep)


SHAPES_2D = [(300, 200), (129, 64), (8, 8), (1030, 136), (64, 1032)]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("bc", [[0, 0], [1, 1], [0, 1], [1, 0]])
@pytest.mark.parametrize("kind,prm,halo", [("jacobi5", [0.2], 1), ("star9r2", [0.1], 2)])
@pytest.mark.parametrize("shape", SHAPES_2D, ids=lambda s: "x".join(map(str, s)))
def test_two_sweeps_2d_bitwise_equal_one_sweep(lope, orc, dtype, bc, kind, prm, halo, shape):
    u0, u0s = to_device(LI.uniform_field(1710, shape), dtype)
    g = lope.Grid(shape, dtype, halo=halo)
    g.set_boundaries(bc)
    st = lope.Stencil.builtin(kind, *prm)
    for T in (2, 5):
        ref = _run(lope, g, st, u0, T, lope.Launch(TMA, 0, 0, 1, -1))
        got = _run(lope, g, st, u0, T, lope.Launch(TMA, 0, 0, 2, -1))
        assert torch.equal(got, ref), T
    assert torch.equal(ref, _run(lope, g, st, u0, 5, lope.Launch(DIRECT, 0, 0, 0, -1)))
    if dtype == "f32" and shape == (300, 200):
        want = orc.apply(u0s, kind, prm, 5, bc=bc)
        G = 1.0 if kind == "jacobi5" else 1.0667
        eps = float(local_eps(kind, prm, [float(np.max(np.abs(u0s))) * G], "f32")[0])
        assert np.max(np.abs(to_host(ref) - want)) <= 5 * G ** 5 * eps


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("bc", [[0, 0], [1, 1], [0, 1], [1, 0]])
@pytest.mark.parametrize("shape", SHAPES_2D, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("kind,prm", [("swe_cgrid", [0.02, 1.0, 1.0]), ("swe_flux", [0.02, 1.0, 0.5, 1.0])])
def test_two_sweeps_2d_three_fields_bitwise_equal_one_sweep(lope, dtype, bc, shape, kind, prm):
    """Shallow water on three fields: the linearised star form and the
    nonlinear flux form (box halo: corner taps, u1 on the ring's corners);
    three fields staged per tile, u1 of each kept on chip; both warp layouts
    of the 32-row tiles."""
    h, u, v = LI.swe_fields(1714, shape)
    eta = kind == "swe_flux" or dtype == "bf16"
    fields = [to_device(x, dtype)[0] for x in (h - 1.0 if eta else h, u, v)]
    g = lope.Grid(shape, dtype, halo=1, nfields=3)
    g.set_boundaries(bc)
    st = lope.Stencil.builtin(kind, *prm)
    for T in (2, 5):
        ref = _run(lope, g, st, fields, T, lope.Launch(TMA, 0, 0, 1, -1))
        for ty in (0, SHORT):
            got = _run(lope, g, st, fields, T, lope.Launch(TMA, 0, ty, 2, -1))
            for k in range(3):
                assert torch.equal(got[k], ref[k]), (T, ty, k)
    direct = _run(lope, g, st, fields, 5, lope.Launch(DIRECT, 0, 0, 0, -1))
    for k in range(3):
        assert torch.equal(direct[k], ref[k]), k


def test_two_sweeps_2d_three_fields_write_only_their_output(lope):
    shape = (300, 200)
    n = int(np.prod(shape))
    guard, sentinel = 4096, -7.0e30
    h, u, v = LI.swe_fields(1715, shape)
    fields = [to_device(x, "f32")[0] for x in (h, u, v)]
    keep = [f.clone() for f in fields]
    st = lope.Stencil.builtin("swe_cgrid", 0.02, 1.0, 1.0)
    for bc in ([0, 0], [1, 1]):
        g = lope.Grid(shape, "f32", halo=1, nfields=3)
        g.set_boundaries(bc)
        bufs = [torch.full((n + 2 * guard,), sentinel, device="cuda") for _ in range(6)]
        views = [b[guard:guard + n].view(shape) for b in bufs]
        _run(lope, g, st, fields, 5, lope.Launch(TMA, 0, 0, 2, -1), out=views[:3], work=views[3:])
        for b in bufs:
            assert bool((b[:guard] == sentinel).all()) and bool((b[guard + n:] == sentinel).all())
        for f, k in zip(fields, keep):
            assert torch.equal(f, k)


def test_two_sweeps_2d_box_tables(lope):
    """Box weight tables of radius 1 and 2 (every corner tap weighted): the
    first sweep fills the corners of its ring."""
    rng = np.random.default_rng(1716)
    shape = (200, 136)
    u0, _ = to_device(LI.uniform_field(1717, shape), "f32")
    for r in (1, 2):
        w = rng.uniform(0.0, 0.08, (2 * r + 1, 2 * r + 1))
        w[r, r] = 1.0 - (w.sum() - w[r, r])
        st = lope.Stencil.linear(w)
        for bc in ([0, 0], [1, 0], [0, 1]):
            g = lope.Grid(shape, "f32", halo=r)
            g.set_boundaries(bc)
            ref = _run(lope, g, st, u0, 6, lope.Launch(DIRECT, 0, 0, 0, -1))
            assert torch.equal(_run(lope, g, st, u0, 6, lope.Launch(TMA, 0, 0, 2, -1)), ref), (r, bc)


def test_two_sweeps_2d_linear_asymmetric_tables(lope):
    rng = np.random.default_rng(1711)
    shape = (200, 136)
    u0, _ = to_device(LI.uniform_field(1712, shape), "f32")
    for r in (1, 2):
        w = np.zeros((2 * r + 1, 2 * r + 1))
        for d in range(2 * r + 1):
            if d != r:
                w[r, d] = rng.uniform(0.01, 0.08)
                w[d, r] = rng.uniform(0.01, 0.08)
        w[r, r] = 1.0 - w.sum()
        st = lope.Stencil.linear(w)
        for bc in ([0, 0], [1, 0]):
            g = lope.Grid(shape, "f32", halo=r)
            g.set_boundaries(bc)
            ref = _run(lope, g, st, u0, 6, lope.Launch(DIRECT, 0, 0, 0, -1))
            assert torch.equal(_run(lope, g, st, u0, 6, lope.Launch(TMA, 0, 0, 2, -1)), ref), (r, bc)


def test_two_sweeps_2d_write_only_their_output(lope):
    shape = (300, 200)
    n = int(np.prod(shape))
    guard, sentinel = 4096, -7.0e30
    u0, _ = to_device(LI.uniform_field(1713, shape), "f32")
    keep = u0.clone()
    st = lope.Stencil.builtin("star9r2", 0.1)
    for bc in ([0, 0], [1, 1]):
        g = lope.Grid(shape, "f32", halo=2)
        g.set_boundaries(bc)
        bufs = [torch.full((n + 2 * guard,), sentinel, device="cuda") for _ in range(2)]
        out, work = (b[guard:guard + n].view(shape) for b in bufs)
        _run(lope, g, st, u0, 5, lope.Launch(TMA, 0, 0, 2, -1), out=out, work=work)
        for b in bufs:
            assert bool((b[:guard] == sentinel).all()) and bool((b[guard + n:] == sentinel).all())
        assert torch.equal(u0, keep)
