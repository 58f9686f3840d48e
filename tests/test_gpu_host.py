"""The host-buffer entry point lope_apply_host: host -> device copy, the
sweeps, device -> host copy on one stream.  Its result must equal lope_apply
on device buffers bitwise, with pinned and with pageable host memory, for
single- and multi-field grids, and calls on two streams must not interfere."""
import numpy as np
import pytest
import torch

import lope_inputs as LI

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pinned", [True, False])
def test_apply_host_equals_device_apply(lope, pinned):
    shape, T = (37, 50, 72), 9
    u = torch.from_numpy(LI.uniform_field(1300, shape).astype(np.float32))
    hin = u.pin_memory() if pinned else u
    hout = torch.empty_like(u).pin_memory() if pinned else torch.empty_like(u)
    g = lope.Grid(shape, "f32", halo=1)
    g.set_boundary(kind="dirichlet", value=0.0)
    st = lope.Stencil.builtin("diff7", 0.1)
    din, dout, dwork = (torch.empty(shape, device="cuda") for _ in range(3))
    s = torch.cuda.Stream()
    lope.apply_host(g, st, hin, hout, din, dout, dwork, nsteps=T, stream=s)
    s.synchronize()
    lope.sync_status()
    ref = lope.apply(g, st, u.cuda(), nsteps=T)
    torch.cuda.synchronize()
    assert torch.equal(hout, ref.cpu())
    assert torch.equal(din.cpu(), u)  # dev_in holds the copied input


def test_apply_host_multi_field_two_streams(lope):
    shape, T = (64, 136), 11
    h, u, v = LI.swe_fields(1301, shape)
    fields = [torch.from_numpy(x.astype(np.float32)).pin_memory() for x in (h - 1.0, u, v)]
    g = lope.Grid(shape, "f32", halo=1, nfields=3)
    st = lope.Stencil.builtin("swe_flux", 0.02, 1.0, 0.5, 1.0)
    outs, streams = [], [torch.cuda.Stream(), torch.cuda.Stream()]
    for s in streams:
        ho = [torch.empty_like(x).pin_memory() for x in fields]
        dev = [[torch.empty(shape, device="cuda") for _ in range(3)] for _ in range(3)]
        lope.apply_host(g, st, fields, ho, dev[0], dev[1], dev[2], nsteps=T, stream=s)
        outs.append((ho, dev))
    torch.cuda.synchronize()
    ref = lope.apply(g, st, [x.cuda() for x in fields], nsteps=T)
    torch.cuda.synchronize()
    for ho, _ in outs:
        for k in range(3):
            assert torch.equal(ho[k], ref[k].cpu()), k


def test_plan_log_one_line_per_distinct_plan(lope, capfd):
    shape = (96, 200)
    u = torch.rand(shape, device="cuda")
    g = lope.Grid(shape, "f32", halo=1)
    g.set_boundaries([1, 0])
    st = lope.Stencil.builtin("jacobi5", 0.2)
    lope.lope_set_option("log", 1)
    try:
        for _ in range(3):
            lope.apply(g, st, u, nsteps=3, launch=lope.Launch(1, 0, 0, 0, -1))
        lope.apply(g, st, u, nsteps=3, launch=lope.Launch(3, 0, 0, 0, -1))
        torch.cuda.synchronize()
    finally:
        lope.lope_set_option("log", 0)
    lope.apply(g, st, u, nsteps=4)  # silent again
    torch.cuda.synchronize()
    lines = [ln for ln in capfd.readouterr().err.splitlines() if ln.startswith("lope: ")]
    assert len(lines) == 2, lines
    assert "grid 96x200 f32 nf=1 bc=[dirichlet,periodic]" in lines[0]
    assert "jacobi5 r=1 euler" in lines[0] and "path=tma" in lines[0]
    assert "launches=3" in lines[0] and "path=direct" in lines[1]


def test_forced_allocation_failure_then_next_call_runs(lope):
    """fail_alloc = 1: the first apply fails with LOPE_ERR_ALLOC before any
    CUDA call and computes nothing; the next apply runs normally."""
    shape = (64, 128)
    u = torch.rand(shape, device="cuda")
    g = lope.Grid(shape, "f32", halo=1)
    st = lope.Stencil.builtin("jacobi5", 0.2)
    ref = lope.apply(g, st, u, nsteps=3)
    torch.cuda.synchronize()
    out = torch.full_like(u, -1.0)
    lope.lope_set_option("fail_alloc", 1)
    try:
        with pytest.raises(lope.LopeError, match="LOPE_ERR_ALLOC"):
            lope.apply(g, st, u, nsteps=3, out=out)
        torch.cuda.synchronize()
        assert bool((out == -1.0).all())
        lope.apply(g, st, u, nsteps=3, out=out)
        torch.cuda.synchronize()
    finally:
        lope.lope_set_option("fail_alloc", 0)
    lope.sync_status()
    assert torch.equal(out, ref)
