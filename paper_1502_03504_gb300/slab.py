"""Slab decomposition of one grid with halo exchange between the slabs.

The paper distributes a halo-annotated array over coarray images as blocks
and refreshes every block's halo from its neighbours with HALO_TRANSFER after
each sweep (Sec. 3.2, Sec. 3.3); its conclusions suggest computing the border
first so that the transfer overlaps the interior (Sec. 5).  Here the grid is
cut along its slowest axis (z in 3D, y in 2D) into slabs, each held in one
buffer with g = R k ghost planes beyond every side that borders another slab
(R the stencil radius, k the sweeps per exchange):

* An exchange copies the first g planes of every slab into the high ghosts of
  its low neighbour and the last g planes into the low ghosts of its high
  neighbour (a periodic axis makes the slabs a ring).
* Then k sweeps run on views of the slab that shrink by R per sweep: sweep s
  updates the planes [-(k-s) R, n + (k-s) R) of the slab, reading R more on
  each side, so after k sweeps the n interior planes are exact without
  another exchange.  A view's sides are EXTERNAL boundaries (the halo is the
  data just beyond it in the buffer) except where the slab ends at the grid's
  own boundary, which keeps the grid's boundary condition.
* Border first: the last sweep of a period computes the g planes at each end
  of the slab first, records an event, and the next exchange of those planes
  starts on a copy stream while the interior planes are computed.

Every sweep runs in the library's kernels (lope_apply on a view grid with
LOPE_BC_EXTERNAL sides); this module plans the views and moves the ghost
planes.  Transports: ``LocalTransport`` (all slabs in this process, copies on
a side stream: device-to-device on one GPU) and ``DistTransport``
(torch.distributed point-to-point, one slab per rank; with NCCL each rank's
ghosts arrive in its own GPU's memory before its kernels read them).
"""
from __future__ import annotations

from dataclasses import dataclass

BC_PERIODIC, BC_DIRICHLET, BC_EXTERNAL = 0, 1, 2


def partition(n: int, parts: int):
    """Split n planes into `parts` contiguous slabs as evenly as possible:
    list of (begin, count), the first n % parts slabs one plane longer."""
    if parts < 1 or parts > n:
        raise ValueError(f"cannot split {n} planes into {parts} slabs")
    q, r = divmod(n, parts)
    out, b = [], 0
    for i in range(parts):
        c = q + (1 if i < r else 0)
        out.append((b, c))
        b += c
    return out


@dataclass(frozen=True)
class View:
    """Planes [begin, begin + count) of a slab (interior coordinates: 0 is the
    slab's first own plane), with the kind of each side: (BC_EXTERNAL, 0.0) or
    the grid's own (kind, value)."""

    begin: int
    count: int
    lo: tuple
    hi: tuple


@dataclass
class Slab:
    index: int      # position along the slowest axis
    begin: int      # first plane in the whole grid
    count: int      # planes owned
    ghost_lo: int   # ghost planes before the owned ones (0 at a grid boundary)
    ghost_hi: int
    low: int        # index of the low neighbour (-1: none)
    high: int       # index of the high neighbour (-1: none)


class SlabPlan:
    """Partition, ghost depth and the per-period sweep views of a grid of
    `n_slow` planes cut into `parts` slabs for a stencil of radius R, k sweeps
    per exchange.  bc_lo / bc_hi: the grid's (kind, value) on the two sides of
    the slowest axis (BC_PERIODIC on both makes the slabs a ring)."""

    def __init__(self, n_slow: int, parts: int, radius: int, k: int, bc_lo, bc_hi):
        if radius < 1 or k < 1:
            raise ValueError("radius and k must be >= 1")
        self.R, self.k, self.g = radius, k, radius * k
        self.bc_lo, self.bc_hi = tuple(bc_lo), tuple(bc_hi)
        periodic = self.bc_lo[0] == BC_PERIODIC and self.bc_hi[0] == BC_PERIODIC
        if (self.bc_lo[0] == BC_PERIODIC) != (self.bc_hi[0] == BC_PERIODIC):
            raise ValueError("a periodic axis is periodic on both sides")
        self.periodic = periodic
        self.slabs = []
        for i, (b, c) in enumerate(partition(n_slow, parts)):
            low = (i - 1) % parts if (i > 0 or periodic) else -1
            high = (i + 1) % parts if (i < parts - 1 or periodic) else -1
            if c < self.g and (low >= 0 or high >= 0):
                raise ValueError(f"slab of {c} planes is thinner than the ghost depth {self.g}")
            self.slabs.append(Slab(i, b, c, self.g if low >= 0 else 0, self.g if high >= 0 else 0,
                                   low, high))

    def extended(self, slab: Slab) -> int:
        """Planes of a slab's buffer: ghosts and owned planes."""
        return slab.ghost_lo + slab.count + slab.ghost_hi

    def sweep_views(self, slab: Slab, s: int):
        """The view(s) of sweep s (1..k) of a period.  The last sweep is split
        border first: the low border, the high border, then the interior."""
        ext = (BC_EXTERNAL, 0.0)
        shrink = (self.k - s) * self.R
        a = -shrink if slab.low >= 0 else 0
        b = slab.count + shrink if slab.high >= 0 else slab.count
        lo = ext if slab.low >= 0 else self.bc_lo
        hi = ext if slab.high >= 0 else self.bc_hi
        if s < self.k or 2 * self.g >= slab.count:
            return [View(a, b - a, lo, hi)]
        g = self.g
        return [View(0, g, lo, ext), View(slab.count - g, g, ext, hi),
                View(g, slab.count - 2 * g, ext, ext)]

    def exchanges(self):
        """Ghost copies of one exchange: (src slab, src first plane, dst slab,
        dst first buffer plane, planes), in buffer coordinates of each slab."""
        out = []
        for s in self.slabs:
            if s.low >= 0:  # my first g planes -> the high ghosts of my low neighbour
                d = self.slabs[s.low]
                out.append((s.index, s.ghost_lo, d.index, d.ghost_lo + d.count, self.g))
            if s.high >= 0:  # my last g planes -> the low ghosts of my high neighbour
                d = self.slabs[s.high]
                out.append((s.index, s.ghost_lo + s.count - self.g, d.index, 0, self.g))
        return out


class LopeSweeper:
    """One sweep of a view with the library's kernels: a lope grid per
    distinct view (slowest-axis extent and sides), lope_apply with nsteps = 1
    on the buffer planes of the view."""

    def __init__(self, lope, stencil, shape, dtype, halo, nfields, boundaries):
        self.L, self.st = lope, stencil
        self.rest = tuple(shape[1:])
        self.dtype, self.halo, self.nf = dtype, halo, nfields
        self.boundaries = boundaries  # (kind, value) per side of the other axes
        self.grids = {}

    def grid(self, view: View):
        key = (view.count, view.lo, view.hi)
        g = self.grids.get(key)
        if g is None:
            g = self.L.Grid((view.count,) + self.rest, self.dtype, halo=self.halo,
                            nfields=self.nf)
            for ax, (lo, hi) in enumerate(self.boundaries, start=1):
                if lo[0] == BC_PERIODIC and hi[0] == BC_PERIODIC:
                    g.set_boundary(ax, -1, BC_PERIODIC)
                else:
                    g.set_boundary(ax, 0, lo[0], lo[1])
                    g.set_boundary(ax, 1, hi[0], hi[1])
            for side, (kind, value) in enumerate((view.lo, view.hi)):
                if kind != BC_PERIODIC:
                    g.set_boundary(0, side, kind, value)
            self.grids[key] = g
        return g

    def __call__(self, view: View, src, dst, first: int, stream=None):
        """src, dst: lists (per field) of slab buffers; first: the buffer plane
        of the view's first plane."""
        g = self.grid(view)
        ins = [x[first:first + view.count] for x in src]
        outs = [x[first:first + view.count] for x in dst]
        self.L.apply(g, self.st, ins if self.nf > 1 else ins[0],
                     out=outs if self.nf > 1 else outs[0], nsteps=1, stream=stream)


class LocalTransport:
    """All slabs in this process: ghost planes copied buffer to buffer (on one
    GPU, device-to-device copies on the copy stream)."""

    def exchange(self, plan: SlabPlan, bufs, local, copy_stream=None):
        import torch

        ctx = torch.cuda.stream(copy_stream) if copy_stream is not None else _nullcontext()
        with ctx:
            for si, sp, di, dp, n in plan.exchanges():
                for f in range(len(bufs[si])):
                    bufs[di][f][dp:dp + n].copy_(bufs[si][f][sp:sp + n], non_blocking=True)


class DistTransport:
    """One slab per rank of a torch.distributed process group: the ghost
    planes go by point-to-point sends and receives (gloo for CPU tensors, NCCL
    for CUDA tensors, where each rank receives into its own device memory)."""

    def __init__(self, group=None):
        self.group = group

    def exchange(self, plan: SlabPlan, bufs, local, copy_stream=None):
        import torch
        import torch.distributed as dist

        me = local[0]
        ops = []
        ctx = torch.cuda.stream(copy_stream) if copy_stream is not None else _nullcontext()
        with ctx:
            recv_bufs = []
            for si, sp, di, dp, n in plan.exchanges():
                for f in range(len(bufs[me])):
                    if si == me and di == me:  # a ring of one slab
                        bufs[me][f][dp:dp + n].copy_(bufs[me][f][sp:sp + n])
                        continue
                    if si == me:
                        src = bufs[me][f][sp:sp + n].contiguous()
                        ops.append(dist.P2POp(dist.isend, src, di, self.group))
                    if di == me:
                        dst = torch.empty_like(bufs[me][f][dp:dp + n])
                        ops.append(dist.P2POp(dist.irecv, dst, si, self.group))
                        recv_bufs.append((bufs[me][f], dp, n, dst))
            if ops:
                for r in dist.batch_isend_irecv(ops):
                    r.wait()
            for buf, dp, n, dst in recv_bufs:
                buf[dp:dp + n].copy_(dst)


class _nullcontext:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


class SlabRunner:
    """Runs a grid decomposed into slabs: owns two buffers per local slab
    (ghosts included), exchanges ghosts every k sweeps and sweeps the views.

    plan: a SlabPlan; local: indices of the slabs held here (all of them with
    LocalTransport, this rank's with DistTransport); sweep: a LopeSweeper (or
    any callable with its signature); alloc(planes, slab) -> list of per-field
    buffers of `planes` planes."""

    def __init__(self, plan: SlabPlan, local, sweep, transport, alloc, streams=None):
        self.plan, self.local, self.sweep, self.transport = plan, list(local), sweep, transport
        self.bufs = [[None, None] for _ in plan.slabs]
        for i in self.local:
            s = plan.slabs[i]
            self.bufs[i] = [alloc(plan.extended(s), s), alloc(plan.extended(s), s)]
        self.cur = 0
        self.streams = streams  # (compute, copy) CUDA streams, or None on the CPU

    def scatter(self, fields):
        """Copy each local slab's planes of the whole-grid fields in."""
        for i in self.local:
            s = self.plan.slabs[i]
            for f, x in enumerate(fields):
                self.bufs[i][self.cur][f][s.ghost_lo:s.ghost_lo + s.count].copy_(
                    x[s.begin:s.begin + s.count])

    def gather(self, fields):
        """Copy each local slab's planes into the whole-grid fields."""
        for i in self.local:
            s = self.plan.slabs[i]
            for f, x in enumerate(fields):
                x[s.begin:s.begin + s.count].copy_(
                    self.bufs[i][self.cur][f][s.ghost_lo:s.ghost_lo + s.count])

    def _state(self, which):
        return [self.bufs[i][which] if i in self.local else None for i in range(len(self.bufs))]

    def run(self, nsteps: int):
        """nsteps sweeps: periods of k sweeps (the last one may be shorter),
        each starting from freshly exchanged ghosts.  The exchange for the next
        period starts on the copy stream as soon as the last sweep's border
        planes are done and overlaps that sweep's interior planes."""
        plan = self.plan
        compute, copy = self.streams if self.streams else (None, None)
        if nsteps <= 0:
            return
        if copy is not None:
            copy.wait_stream(compute)
        self.transport.exchange(plan, self._state(self.cur), self.local, copy)
        done = 0
        while done < nsteps:
            k = min(plan.k, nsteps - done)
            done += k
            if compute is not None:
                compute.wait_stream(copy)  # the ghosts of this period are in
            for s in range(plan.k - k + 1, plan.k + 1):
                src, dst = self.cur, 1 - self.cur
                views = {i: plan.sweep_views(plan.slabs[i], s) for i in self.local}
                for i in self.local:  # every view but a last-sweep interior
                    for v in views[i][:2]:
                        self._sweep(i, v, src, dst, compute)
                if s == plan.k and done < nsteps:
                    # border planes done: start the next exchange beside the interior
                    if copy is not None:
                        copy.wait_stream(compute)
                    interior = [(i, views[i][2:]) for i in self.local]
                    self.cur = dst
                    self.transport.exchange(plan, self._state(dst), self.local, copy)
                    for i, rest in interior:
                        for v in rest:
                            self._sweep(i, v, src, dst, compute)
                else:
                    for i in self.local:
                        for v in views[i][2:]:
                            self._sweep(i, v, src, dst, compute)
                    self.cur = dst
        if compute is not None:
            compute.wait_stream(copy)

    def _sweep(self, i, view, src, dst, compute):
        slab = self.plan.slabs[i]
        self.sweep(view, self.bufs[i][src], self.bufs[i][dst], slab.ghost_lo + view.begin,
                   compute.cuda_stream if compute is not None else None)
