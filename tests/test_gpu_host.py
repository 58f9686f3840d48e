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
