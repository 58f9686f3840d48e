"""Both compiled tile heights of the TMA kernels give bitwise the same result.

The runner picks tall tiles on large grids and short ones on small grids
(lope_launch.tile_y 1 / 2 forces short / tall on the TMA path).  Every local
function evaluates the same arithmetic on any tiling, so forced tall, forced
short and the direct kernel must agree bitwise on grids with ragged edge tiles
in every axis and with periodic and Dirichlet boundaries; one case per shape is
also checked against the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import lope_inputs as LI
from gpu_helpers import bound_f32, to_device, to_host

pytestmark = pytest.mark.gpu

SHORT, TALL = 1, 2


def _run(L, g, st, fields, T, launch):
    out = L.apply(g, st, fields, nsteps=T, launch=launch)
    torch.cuda.synchronize()
    L.sync_status()
    return out if isinstance(out, list) else [out]


def _check(L, g, st, fields, T):
    tall = _run(L, g, st, fields, T, L.Launch(1, 0, TALL, 0, -1))
    short = _run(L, g, st, fields, T, L.Launch(1, 0, SHORT, 0, -1))
    direct = _run(L, g, st, fields, T, L.Launch(3, 0, 0, 0, -1))
    for k in range(len(tall)):
        assert torch.equal(tall[k], short[k]), k
        assert torch.equal(tall[k], direct[k]), k
    return tall


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("bc", [[0, 0], [1, 0], [0, 1]])
@pytest.mark.parametrize("kind,prm,halo", [("jacobi5", [0.2], 1), ("star9r2", [0.1], 2)])
def test_2d_single_field_tall_short_direct(lope, orc, dtype, bc, kind, prm, halo):
    shape, T = (300, 200), 5  # 3 tall tiles (the last ragged) x 4 columns (ragged)
    u0, u0s = to_device(LI.uniform_field(1500, shape), dtype)
    g = lope.Grid(shape, dtype, halo=halo)
    g.set_boundaries(bc)
    st = lope.Stencil.builtin(kind, *prm)
    out = _check(lope, g, st, u0, T)
    if dtype == "f32":
        want = orc.apply(u0s, kind, prm, T, bc=bc)
        G = 1.0 if kind == "jacobi5" else abs(1 - 5 * prm[0]) + prm[0] * (4 * 4 / 3 + 4 / 12)
        assert np.max(np.abs(to_host(out[0]) - want)) <= bound_f32(T, 1.0, 12, G)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("bc", [[1, 1, 1], [0, 0, 0], [1, 0, 1]])
def test_3d_tall_short_direct(lope, orc, dtype, bc):
    shape, T = (40, 150, 136), 4  # 3 tall tile rows (the last ragged), 3 columns (ragged)
    u0, u0s = to_device(LI.uniform_field(1501, shape), dtype)
    g = lope.Grid(shape, dtype, halo=1)
    g.set_boundaries(bc)
    st = lope.Stencil.builtin("diff7", 0.1)
    out = _check(lope, g, st, u0, T)
    if dtype == "f32":
        want = orc.apply(u0s, "diff7", [0.1], T, bc=bc)
        assert np.max(np.abs(to_host(out[0]) - want)) <= bound_f32(T, 1.0, 9)


@pytest.mark.parametrize("kind,prm", [("swe_flux", [0.02, 1.0, 0.5, 1.0]),
                                      ("swe_cgrid", [0.02, 1.0, 1.0])])
@pytest.mark.parametrize("bc", [[0, 0], [1, 1]])
def test_2d_multi_field_tall_short_direct(lope, kind, prm, bc):
    shape, T = (150, 200), 4
    h, u, v = LI.swe_fields(1502, shape)
    fields = [to_device(x, "f32")[0] for x in ((h - 1.0) if kind == "swe_flux" else h, u, v)]
    g = lope.Grid(shape, "f32", halo=1, nfields=3)
    g.set_boundaries(bc)
    _check(lope, g, lope.Stencil.builtin(kind, *prm), fields, T)
