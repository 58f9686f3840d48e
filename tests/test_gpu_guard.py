"""Out-of-bounds write detection: every kernel path writes only its output.

Each output and work buffer is a view into a larger allocation whose guard
bands before and after the view hold a sentinel bit pattern.  After the run
the guards must be unchanged, and the input must be unchanged.  Paths: TMA 2D
(short and tall tiles, star and box functions), TMA 3D z-march, trapezoid,
direct, the Runge-Kutta stage and fused forms, the batched kernel, a run-time
compiled function, and the host-buffer entry point.
"""
import numpy as np
import pytest
import torch

import lope_inputs as LI

pytestmark = pytest.mark.gpu

GUARD = 4096  # elements on each side of every view
SENTINEL = -7.0e30


def _guarded(shape, dtype):
    n = int(np.prod(shape))
    buf = torch.full((n + 2 * GUARD,), SENTINEL, dtype=dtype, device="cuda")
    return buf, buf[GUARD:GUARD + n].view(shape)


def _guards_intact(buf, n):
    want = torch.full((GUARD,), SENTINEL, dtype=buf.dtype, device=buf.device)
    return torch.equal(buf[:GUARD], want) and torch.equal(buf[GUARD + n:], want)


def _check(L, g, st, ins, nsteps, launch, work_states=1):
    shape = tuple(ins[0].shape)
    n = int(np.prod(shape))
    outs, works, bufs = [], [], []
    for x in ins:
        b, v = _guarded(shape, x.dtype)
        bufs.append((b, n))
        outs.append(v)
        b, v = _guarded((work_states,) + shape, x.dtype)
        bufs.append((b, n * work_states))
        works.append(v if work_states > 1 else v[0])
    keep = [x.clone() for x in ins]
    L.apply(g, st, ins if len(ins) > 1 else ins[0], out=outs, work=works, nsteps=nsteps,
            launch=launch)
    torch.cuda.synchronize()
    L.sync_status()
    for b, m in bufs:
        assert _guards_intact(b, m), launch
    for x, k in zip(ins, keep):
        assert torch.equal(x, k)


CASES_2D = [("jacobi5", [0.2], 1, 1), ("star9r2", [0.1], 2, 1), ("swe_flux", [0.02, 1.0, 0.5, 1.0], 1, 3)]


@pytest.mark.parametrize("kind,prm,halo,nf", CASES_2D)
@pytest.mark.parametrize("bc", [[0, 0], [1, 1]])
def test_2d_paths_write_only_their_output(lope, kind, prm, halo, nf, bc):
    shape = (150, 200)
    ins = [torch.from_numpy(LI.uniform_field(1700 + f, shape).astype(np.float32)).cuda()
           for f in range(nf)]
    g = lope.Grid(shape, "f32", halo=halo, nfields=nf)
    g.set_boundaries(bc)
    st = lope.Stencil.builtin(kind, *prm)
    for launch in (lope.Launch(1, 0, 1, 0, -1), lope.Launch(1, 0, 2, 0, -1),
                   lope.Launch(2, 64, 32, 3, -1), lope.Launch(3, 0, 0, 0, -1)):
        _check(lope, g, st, ins, 5, launch)
    st.set_scheme("rk3")
    for launch in (lope.Launch(1, 0, 0, 0, -1), lope.Launch(2, 64, 16, 2, -1),
                   lope.Launch(3, 0, 0, 0, -1)):
        _check(lope, g, st, ins, 3, launch, work_states=2)


@pytest.mark.parametrize("bc", [[0, 0, 0], [1, 1, 1]])
def test_3d_paths_write_only_their_output(lope, bc):
    shape = (40, 70, 136)
    u = torch.from_numpy(LI.uniform_field(1710, shape).astype(np.float32)).cuda()
    g = lope.Grid(shape, "f32", halo=1)
    g.set_boundaries(bc)
    st = lope.Stencil.builtin("diff7", 0.1)
    for launch in (lope.Launch(1, 0, 1, 0, -1), lope.Launch(1, 0, 2, 0, -1),
                   lope.Launch(3, 0, 0, 0, -1)):
        _check(lope, g, st, [u], 4, launch)


def test_batched_and_source_and_host_paths_write_only_their_output(lope):
    # batched: guarded outputs and work buffers for three grids
    shapes = [(70, 130), (33, 257), (128, 64)]
    grids, ins, outs, works, bufs = [], [], [], [], []
    for i, s in enumerate(shapes):
        g = lope.Grid(s, "f32", halo=1)
        g.set_boundaries([i % 2, i % 2])
        grids.append(g)
        ins.append(torch.from_numpy(LI.uniform_field(1720 + i, s).astype(np.float32)).cuda())
        for lst in (outs, works):
            b, v = _guarded(s, torch.float32)
            bufs.append((b, int(np.prod(s))))
            lst.append(v)
    st = lope.Stencil.builtin("jacobi5", 0.2)
    lope.apply_batch(grids, st, ins, outs, works, nsteps=9, launch=lope.Launch(2, 128, 32, 4, -1))
    torch.cuda.synchronize()
    lope.sync_status()
    assert all(_guards_intact(b, m) for b, m in bufs)
    # a run-time compiled function with corner taps
    body = "out[0] = fma_(P[0], sub(add(U(0, 1, 1), U(0, -1, -1)), mul(C(2), U(0, 0, 0))), U(0, 0, 0));"
    src = lope.Stencil.source(body, ndim=2, radius=1, params=[0.1], box=True)
    g = lope.Grid((150, 200), "f32", halo=1)
    u = torch.from_numpy(LI.uniform_field(1730, (150, 200)).astype(np.float32)).cuda()
    for launch in (lope.Launch(1, 0, 0, 0, -1), lope.Launch(2, 64, 32, 2, -1), lope.Launch(3, 0, 0, 0, -1)):
        _check(lope, g, src, [u], 4, launch)
    # the host-buffer entry point: guarded device buffers
    hin = u.cpu().pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    dbufs = [_guarded((150, 200), torch.float32) for _ in range(3)]
    lope.apply_host(g, lope.Stencil.builtin("jacobi5", 0.2), hin, hout, dbufs[0][1], dbufs[1][1],
                    dbufs[2][1], nsteps=6)
    torch.cuda.synchronize()
    assert all(_guards_intact(b, 150 * 200) for b, _ in dbufs)


@pytest.mark.parametrize("bc", [[0, 0, 0], [1, 0, 1]])
def test_unaligned_paths_write_only_their_output(lope, bc):
    # rows whose pitch is not a multiple of 16 bytes: 2D trapezoid tiles fusing
    # 4 sweeps (the default) and the 3D plane march and direct kernel
    u2 = torch.from_numpy(LI.uniform_field(1740, (83, 261)).astype(np.float32)).cuda()
    g2 = lope.Grid((83, 261), "f32", halo=1)
    g2.set_boundaries(bc[1:])
    st2 = lope.Stencil.builtin("jacobi5", 0.2)
    for launch in (lope.Launch(0, 0, 0, 0, -1), lope.Launch(2, 64, 16, 4, -1)):
        _check(lope, g2, st2, [u2], 9, launch)
    u3 = torch.from_numpy(LI.uniform_field(1741, (21, 19, 45)).astype(np.float32)).cuda()
    g3 = lope.Grid((21, 19, 45), "f32", halo=1)
    g3.set_boundaries(bc)
    st3 = lope.Stencil.builtin("diff7", 0.1)
    for launch in (lope.Launch(4, 0, 0, 0, -1), lope.Launch(3, 0, 0, 0, -1)):
        _check(lope, g3, st3, [u3], 5, launch)
