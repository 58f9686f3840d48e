"""Slab decomposition with halo exchange, host logic on the CPU.

The plan (partition, ghost depth, shrinking sweep views, border-first split,
exchange list) is checked directly.  The runner is then driven with CPU
tensors and a sweep done by the FP64 oracle on each view's planes plus its
external halo (the view's own boundary elsewhere), so the partition, the
ghost exchange and the view bookkeeping are checked against the whole-domain
oracle: in one process (three slabs, copies between their buffers) and as
two gloo ranks exchanging ghost planes point to point.  The kernels' reading
of an external halo is checked on the GPU (test_gpu_slab.py).
"""
import os

import numpy as np
import pytest
import torch

import lope_inputs as LI
from paper_1502_03504_gb300.slab import (BC_DIRICHLET, BC_EXTERNAL, BC_PERIODIC, DistTransport,
                                         LocalTransport, SlabPlan, SlabRunner, View, partition)


def test_partition_is_contiguous_and_balanced():
    assert partition(10, 3) == [(0, 4), (4, 3), (7, 3)]
    assert partition(8, 8) == [(i, 1) for i in range(8)]
    for n, p in ((513, 7), (64, 2), (100, 1)):
        parts = partition(n, p)
        assert sum(c for _, c in parts) == n and parts[0][0] == 0
        assert all(b2 == b1 + c1 for (b1, c1), (b2, _) in zip(parts, parts[1:]))
        assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    with pytest.raises(ValueError):
        partition(3, 4)


def test_plan_views_shrink_and_exchanges_pair_up():
    plan = SlabPlan(40, 3, radius=2, k=3, bc_lo=(BC_DIRICHLET, 0.5), bc_hi=(BC_DIRICHLET, 0.0))
    assert plan.g == 6
    s0, s1, s2 = plan.slabs
    assert (s0.ghost_lo, s0.ghost_hi, s1.ghost_lo, s1.ghost_hi, s2.ghost_hi) == (0, 6, 6, 6, 0)
    ext = (BC_EXTERNAL, 0.0)
    # middle slab: sweep 1 covers R (k-1) = 4 ghost planes on each side
    assert plan.sweep_views(s1, 1) == [View(-4, s1.count + 8, ext, ext)]
    assert plan.sweep_views(s1, 2) == [View(-2, s1.count + 4, ext, ext)]
    # last sweep: low border, high border, interior
    v = plan.sweep_views(s1, 3)
    assert v == [View(0, 6, ext, ext), View(s1.count - 6, 6, ext, ext),
                 View(6, s1.count - 12, ext, ext)]
    # the first slab keeps the grid's own low boundary
    assert plan.sweep_views(s0, 1)[0] == View(0, s0.count + 4, (BC_DIRICHLET, 0.5), ext)
    ex = plan.exchanges()
    assert (0, s0.count - 6, 1, 0, 6) in ex and (1, 6, 0, s0.count, 6) in ex
    assert len(ex) == 4
    ring = SlabPlan(40, 2, radius=1, k=2, bc_lo=(BC_PERIODIC, 0.0), bc_hi=(BC_PERIODIC, 0.0))
    assert all(s.low >= 0 and s.high >= 0 for s in ring.slabs) and len(ring.exchanges()) == 4
    with pytest.raises(ValueError):
        SlabPlan(10, 4, radius=2, k=2, bc_lo=(BC_DIRICHLET, 0.0), bc_hi=(BC_DIRICHLET, 0.0))


class OracleSweeper:
    """One sweep of a view by the FP64 oracle: the view's planes plus R planes
    beyond each external side, swept with the view's boundaries (what lies
    past the external planes does not reach the kept planes in one sweep)."""

    def __init__(self, orc, kind, prm, other_bc, R):
        self.orc, self.kind, self.prm, self.other_bc, self.R = orc, kind, prm, other_bc, R

    def __call__(self, view, src, dst, first, stream=None):
        lo = self.R if view.lo[0] == BC_EXTERNAL else 0
        hi = self.R if view.hi[0] == BC_EXTERNAL else 0
        ext = [x[first - lo:first + view.count + hi].numpy() for x in src]
        kind = [BC_DIRICHLET if s[0] == BC_EXTERNAL else s[0] for s in (view.lo, view.hi)]
        val = [0.0 if s[0] == BC_EXTERNAL else s[1] for s in (view.lo, view.hi)]
        out = self.orc.apply(ext if len(ext) > 1 else ext[0], self.kind, self.prm, 1,
                             bc=[tuple(kind)] + self.other_bc, bval=[tuple(val)] + [0.0] * len(
                                 self.other_bc))
        out = out if len(ext) > 1 else [out]
        for f, y in enumerate(out):
            dst[f][first:first + view.count] = torch.from_numpy(y[lo:lo + view.count])


def _alloc(rest, nf):
    return lambda planes, slab: [torch.full((planes,) + rest, float("nan"), dtype=torch.float64)
                                 for _ in range(nf)]


CASES = [  # kind, prm, shape, R, slow-axis bc (lo, hi), other axes' bc
    ("jacobi5", [0.2], (37, 24), 1, ((BC_DIRICHLET, 0.25), (BC_DIRICHLET, -0.5)), [0]),
    ("star9r2", [0.1], (41, 20), 2, ((BC_PERIODIC, 0.0), (BC_PERIODIC, 0.0)), [0]),
    ("diff7", [0.1], (30, 9, 12), 1, ((BC_DIRICHLET, 0.0), (BC_DIRICHLET, 0.0)), [1, 0]),
    ("swe_flux", [0.02, 1.0, 0.5, 1.0], (33, 16), 1, ((BC_PERIODIC, 0.0), (BC_PERIODIC, 0.0)),
     [0]),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
@pytest.mark.parametrize("k", [1, 2])
def test_local_slabs_match_whole_domain_oracle(orc, case, k):
    kind, prm, shape, R, (blo, bhi), other = case
    nf = 3 if kind.startswith("swe") else 1
    T = 5
    fields = [LI.uniform_field(1800 + f, shape) * (0.1 if nf > 1 else 1.0) for f in range(nf)]
    slow_bc = (blo[0], bhi[0]) if blo[0] != BC_PERIODIC else 0
    slow_val = (blo[1], bhi[1])
    want = orc.apply(fields if nf > 1 else fields[0], kind, prm, T, bc=[slow_bc] + other,
                     bval=[slow_val] + [0.0] * len(other))
    want = want if nf > 1 else [want]
    plan = SlabPlan(shape[0], 3, R, k, blo, bhi)
    runner = SlabRunner(plan, range(3), OracleSweeper(orc, kind, prm, other, R), LocalTransport(),
                        _alloc(shape[1:], nf))
    runner.scatter([torch.from_numpy(f) for f in fields])
    runner.run(T)
    got = [torch.zeros(shape, dtype=torch.float64) for _ in range(nf)]
    runner.gather(got)
    for f in range(nf):
        assert np.max(np.abs(got[f].numpy() - want[f])) <= 1e-14 * max(1.0, np.max(np.abs(want[f])))


def _rank_main(rank, world, port, kind, prm, shape, R, k, blo, bhi, other, T, result_path):
    import torch.distributed as dist

    import oracle as orc

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nf = 3 if kind.startswith("swe") else 1
        fields = [LI.uniform_field(1900 + f, shape) * (0.1 if nf > 1 else 1.0) for f in range(nf)]
        plan = SlabPlan(shape[0], world, R, k, blo, bhi)
        runner = SlabRunner(plan, [rank], OracleSweeper(orc, kind, prm, other, R),
                            DistTransport(), _alloc(shape[1:], nf))
        runner.scatter([torch.from_numpy(f) for f in fields])
        runner.run(T)
        part = [torch.zeros(shape, dtype=torch.float64) for _ in range(nf)]
        runner.gather(part)  # only this rank's planes are filled
        for f in range(nf):
            dist.all_reduce(part[f])
        if rank == 0:
            np.save(result_path, np.stack([p.numpy() for p in part]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[3]], ids=lambda c: c[0])
def test_two_gloo_ranks_exchange_ghosts_and_match_whole_domain(orc, tmp_path, case):
    import socket

    import torch.multiprocessing as mp

    kind, prm, shape, R, (blo, bhi), other = case
    nf = 3 if kind.startswith("swe") else 1
    T, k = 6, 2
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "field.npy")
    mp.start_processes(_rank_main, args=(2, port, kind, prm, shape, R, k, blo, bhi, other, T, out),
                       nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    fields = [LI.uniform_field(1900 + f, shape) * (0.1 if nf > 1 else 1.0) for f in range(nf)]
    slow_bc = (blo[0], bhi[0]) if blo[0] != BC_PERIODIC else 0
    want = orc.apply(fields if nf > 1 else fields[0], kind, prm, T, bc=[slow_bc] + other,
                     bval=[(blo[1], bhi[1])] + [0.0] * len(other))
    want = want if nf > 1 else [want]
    for f in range(nf):
        assert np.max(np.abs(got[f] - want[f])) <= 1e-14 * max(1.0, np.max(np.abs(want[f])))
