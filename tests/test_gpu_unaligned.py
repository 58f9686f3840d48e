"""Grids whose row pitch is not a multiple of 16 bytes (no TMA staging).

The planner sends such 2D grids to trapezoid tiles fusing 4 sweeps (128 x 32
for one field, 64 x 16 for several) and 3D grids to the plane march (launch
path 4), which is checked against the direct kernel.  Every
path evaluates the same arithmetic, so the default plan, trapezoid tiles with
one sweep and the direct kernel agree bitwise; FP64 runs match the oracle
(normwise 1e-12).
"""
import numpy as np
import pytest
import torch

import lope_inputs as LI
from gpu_helpers import normwise, to_device, to_host

pytestmark = pytest.mark.gpu

FLUX = [0.02, 1.0, 0.5, 1.0]
CASES_2D = [("jacobi5", [0.2], 1, 1), ("star9r2", [0.1], 2, 1), ("swe_cgrid", [0.02, 1.0, 1.0], 1, 3),
            ("swe_flux", FLUX, 1, 3)]


def _fields(kind, shape, seed, nf):
    if kind.startswith("swe"):
        h, u, v = LI.swe_fields(seed, shape)
        return [h - 1.0, u, v]
    return [LI.uniform_field(seed + f, shape) for f in range(nf)]


def _run(L, g, st, fields, T, launch=None):
    out = L.apply(g, st, fields, nsteps=T, launch=launch)
    torch.cuda.synchronize()
    L.sync_status()
    return out if isinstance(out, list) else [out]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("bc", [[0, 0], [1, 0], [1, 1]])
@pytest.mark.parametrize("kind,prm,halo,nf", CASES_2D)
def test_2d_default_trapezoid_direct_bitwise(lope, dtype, bc, kind, prm, halo, nf):
    shape, T = (83, 261), 9  # 261 * 4 B and 261 * 2 B are not multiples of 16
    fl = [to_device(f, dtype)[0] for f in _fields(kind, shape, 1400, nf)]
    g = lope.Grid(shape, dtype, halo=halo, nfields=nf)
    g.set_boundaries(bc)
    st = lope.Stencil.builtin(kind, *prm)
    ref = _run(lope, g, st, fl, T)
    for launch in (lope.Launch(3, 0, 0, 0, -1), lope.Launch(2, 64, 32, 1, -1),
                   lope.Launch(2, 128, 32, 4, -1), lope.Launch(2, 64, 16, 4, 0)):
        got = _run(lope, g, st, fl, T, launch)
        for k in range(nf):
            assert torch.equal(got[k], ref[k]), (launch, k)


@pytest.mark.parametrize("kind,prm,halo,nf", CASES_2D)
def test_2d_fp64_odd_width_vs_oracle(lope, orc, kind, prm, halo, nf):
    shape, T = (67, 133), 10
    fl = _fields(kind, shape, 1410, nf)
    dev, stored = zip(*(to_device(f, "f64") for f in fl))
    g = lope.Grid(shape, "f64", halo=halo, nfields=nf)
    g.set_boundaries([0, 1])
    st = lope.Stencil.builtin(kind, *prm)
    want = orc.apply(list(stored) if nf > 1 else stored[0], kind, prm, T, bc=[0, 1])
    want = want if nf > 1 else [want]
    for launch in (None, lope.Launch(3, 0, 0, 0, -1)):
        got = _run(lope, g, st, list(dev), T, launch)
        for k in range(nf):
            assert normwise(to_host(got[k]), want[k]) <= 1e-12, (launch, k)


@pytest.mark.parametrize("bc", [[0, 0, 0], [1, 1, 1], [1, 0, 1]])
def test_3d_direct_odd_width(lope, orc, bc):
    shape, T = (19, 23, 37), 6
    u64, u64s = to_device(LI.uniform_field(1420, shape), "f64")
    g = lope.Grid(shape, "f64", halo=1)
    g.set_boundaries(bc)
    st = lope.Stencil.builtin("diff7", 0.1)
    got = _run(lope, g, st, u64, T)[0]
    assert normwise(to_host(got), orc.apply(u64s, "diff7", [0.1], T, bc=bc)) <= 1e-12
    u32, _ = to_device(LI.uniform_field(1420, shape), "f32")
    g32 = lope.Grid(shape, "f32", halo=1)
    g32.set_boundaries(bc)
    a = _run(lope, g32, st, u32, T)[0]
    b = _run(lope, g32, st, u32, T, lope.Launch(3, 0, 0, 0, 1))[0]
    assert torch.equal(a, b)


def test_direct_wide_and_narrow_rows(lope, orc):
    # rows of several 256-point units and rows narrower than the radius box
    for shape in ((5, 1031), (300, 3), (2, 2, 600)):
        u, us = to_device(LI.uniform_field(1430, shape), "f64")
        g = lope.Grid(shape, "f64", halo=1)
        g.set_boundaries([0] * len(shape))
        kind = "diff7" if len(shape) == 3 else "jacobi5"
        st = lope.Stencil.builtin(kind, 0.1)
        got = _run(lope, g, st, u, 4, lope.Launch(3, 0, 0, 0, -1))[0]
        assert normwise(to_host(got), orc.apply(us, kind, [0.1], 4, bc=[0] * len(shape))) <= 1e-12, shape


MARCH, DIRECT = 4, 3


# 45 and 131 points per row: no TMA staging for any storage type.  The second
# shape spans several column tiles with ragged tails and four z chunks, each
# refilling its plane ring from its own first planes.  205 and 206 points per
# row give the copied-plane z-march tiles whose boxes lie inside the grid, with
# rows starting at every 4-byte (205) or 8-byte (206) offset: 16-, 8- and
# 4-byte copies.
@pytest.mark.parametrize("shape", [(21, 19, 45), (70, 37, 131), (12, 70, 205), (9, 67, 206)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("bc", [[0, 0, 0], [1, 1, 1], [0, 1, 0], [1, 0, 1]])
def test_3d_march_equals_direct(lope, dtype, bc, shape):
    T = 5
    u, _ = to_device(LI.uniform_field(1440, shape), dtype)
    rng = np.random.default_rng(1441)
    box = rng.uniform(-0.1, 0.1, (3, 3, 3))
    star2 = np.zeros((5, 5, 5))
    star2[2, 2, :] = star2[2, :, 2] = star2[:, 2, 2] = rng.uniform(-0.1, 0.1, 5)
    for st, halo in ((lope.Stencil.builtin("diff7", 0.1), 1), (lope.Stencil.linear(box), 1),
                     (lope.Stencil.linear(star2), 2), (lope.Stencil.builtin("diff7", 0.1).set_scheme("rk3"), 1)):
        g = lope.Grid(shape, dtype, halo=halo)
        bval = [0.0, 0.0, 0.0] if dtype == "bf16" else [(0.5, -0.3), -0.25, (1.0, 0.2)]
        g.set_boundaries(bc, bval)
        b = _run(lope, g, st, u, T, lope.Launch(DIRECT, 0, 0, 0, -1))[0]
        for ty in (0, 1):  # the march's default tiles, and its short tiles
            a = _run(lope, g, st, u, T, lope.Launch(MARCH, 0, ty, 0, -1))[0]
            assert torch.equal(a, b), (st.scheme, halo, ty)


def test_3d_odd_width_default_is_march_and_matches_oracle(lope, orc, capfd):
    shape, T = (33, 18, 27), 8
    u, us = to_device(LI.uniform_field(1450, shape), "f64")
    g = lope.Grid(shape, "f64", halo=1)
    g.set_boundaries([1, 0, 1], [0.25, 0.0, -0.5])
    st = lope.Stencil.builtin("diff7", 0.1)
    lope.lope_set_option("log", 1)
    try:
        got = _run(lope, g, st, u, T)[0]
    finally:
        lope.lope_set_option("log", 0)
    assert "path=march" in capfd.readouterr().err
    want = orc.apply(us, "diff7", [0.1], T, bc=[1, 0, 1], bval=[0.25, 0.0, -0.5])
    assert normwise(to_host(got), want) <= 1e-12
    direct = _run(lope, g, st, u, T, lope.Launch(DIRECT, 0, 0, 0, -1))[0]
    assert normwise(to_host(direct), want) <= 1e-12


def test_box_corners_across_dirichlet_sides_vs_oracle(lope, orc):
    """Box stencils read corner ghosts that cross several Dirichlet sides with
    different values: the slowest crossed axis decides, on every path."""
    rng = np.random.default_rng(1460)
    shape3, T = (9, 11, 13), 3
    u3, u3s = to_device(LI.uniform_field(1461, shape3), "f64")
    w3 = rng.uniform(-0.05, 0.05, (3, 3, 3))
    bc3, bv3 = [1, 1, 1], [(0.7, -0.2), (0.5, 0.1), (-0.3, 0.9)]
    g3 = lope.Grid(shape3, "f64", halo=1)
    g3.set_boundaries(bc3, bv3)
    st3 = lope.Stencil.linear(w3)
    want3 = orc.apply(u3s, "linear", nsteps=T, bc=bc3, bval=bv3, weights_table=w3)
    for launch in (lope.Launch(MARCH, 0, 0, 0, -1), lope.Launch(DIRECT, 0, 0, 0, -1)):
        got = _run(lope, g3, st3, u3, T, launch)[0]
        assert normwise(to_host(got), want3) <= 1e-12, launch
    shape2 = (37, 41)
    u2, u2s = to_device(LI.uniform_field(1462, shape2), "f64")
    w2 = rng.uniform(-0.1, 0.1, (3, 3))
    bc2, bv2 = [1, 1], [(0.5, 0.1), (-0.3, 0.9)]
    g2 = lope.Grid(shape2, "f64", halo=1)
    g2.set_boundaries(bc2, bv2)
    st2 = lope.Stencil.linear(w2)
    want2 = orc.apply(u2s, "linear", nsteps=T, bc=bc2, bval=bv2, weights_table=w2)
    for launch in (None, lope.Launch(2, 32, 8, 3, -1), lope.Launch(DIRECT, 0, 0, 0, -1)):
        got = _run(lope, g2, st2, u2, T, launch)[0]
        assert normwise(to_host(got), want2) <= 1e-12, launch
