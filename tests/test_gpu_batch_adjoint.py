"""GPU parity of the batched persistent launch and of the adjoint.

Batched: every grid of the batch against the FP64 oracle, and bitwise against
the same grid advanced alone by the per-grid trapezoid kernel (same tile
arithmetic).  Adjoint: the discrete adjoint of the oracle (FP64, 1e-12),
central finite differences of the oracle's FP64 loss, checkpoint-interval
independence, the dot-product identity at full size, and the autograd
binding.
"""
import numpy as np
import pytest
import torch

import lope_inputs as LI
from error_bounds import local_eps
from gpu_helpers import bound_f32, normwise, to_device, to_host

pytestmark = pytest.mark.gpu


def _batch_setup(lope, shapes, kinds, dtype, seed):
    grids, ins, stored = [], [], []
    off = 0
    for (ny, nx), k in zip(shapes, kinds):
        g = lope.Grid((ny, nx), dtype, halo=1)
        g.set_boundaries([k, k])
        u = LI.uniform(seed, ny * nx, off).reshape(ny, nx)
        off += ny * nx
        t, s = to_device(u, dtype)
        grids.append(g)
        ins.append(t)
        stored.append(s)
    return grids, ins, stored


@pytest.mark.parametrize("k", [1, 3, 4])
def test_batch_small_vs_oracle_and_per_grid(lope, orc, k):
    shapes, kinds = LI.batch_shapes(77, 14, lo=9, hi=300)
    shapes[0] = (1, 5)  # degenerate single-row grid
    grids, ins, stored = _batch_setup(lope, shapes, kinds, "f32", 78)
    st = lope.Stencil.builtin("jacobi5", 0.2)
    T = 7
    launch = lope.Launch(2, 64, 32, k, -1)
    outs = lope.apply_batch(grids, st, ins, nsteps=T, launch=launch)
    torch.cuda.synchronize()
    lope.sync_status()
    for g, i, o, s, kind in zip(grids, ins, outs, stored, kinds):
        want = orc.apply(s, "jacobi5", [0.2], T, bc=[kind, kind])
        assert np.max(np.abs(to_host(o) - want)) <= bound_f32(T, 1.0, 7)
        alone = lope.apply(g, st, i, nsteps=T, launch=launch)
        torch.cuda.synchronize()
        assert torch.equal(alone, o)


def test_batch_graph_replay_reads_live_buffers(lope):
    shapes, kinds = LI.batch_shapes(79, 6, lo=30, hi=200)
    grids, ins, _ = _batch_setup(lope, shapes, kinds, "f32", 80)
    st = lope.Stencil.builtin("jacobi5", 0.2)
    outs = [torch.empty_like(t) for t in ins]
    works = [torch.empty_like(t) for t in ins]
    ws = torch.empty(lope.batch_workspace_size(grids, st), dtype=torch.uint8, device="cuda")
    launch = lope.Launch(2, 64, 16, 2, -1)
    lope.apply_batch(grids, st, ins, outs, works, 5, launch, ws)
    first = [o.clone() for o in outs]
    lope.apply_batch(grids, st, ins, outs, works, 5, launch, ws)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(first, outs))
    for t in ins:
        t.mul_(0.5)
    lope.apply_batch(grids, st, ins, outs, works, 5, launch, ws)
    torch.cuda.synchronize()
    for g, i, o in zip(grids, ins, outs):
        assert torch.equal(lope.apply(g, st, i, nsteps=5, launch=launch), o)


def test_batch_bf16_and_fp64(lope, orc):
    shapes, kinds = LI.batch_shapes(81, 5, lo=16, hi=130)
    for dtype, tol in (("f64", 1e-12), ("bf16", None)):
        grids, ins, stored = _batch_setup(lope, shapes, kinds, dtype, 82)
        st = lope.Stencil.builtin("jacobi5", 0.2)
        outs = lope.apply_batch(grids, st, ins, nsteps=6, launch=lope.Launch(2, 32, 16, 3, -1))
        torch.cuda.synchronize()
        for o, s, kind in zip(outs, stored, kinds):
            want = orc.apply(s, "jacobi5", [0.2], 6, bc=[kind, kind])
            if dtype == "f64":
                assert normwise(to_host(o), want) <= tol
            else:
                assert np.max(np.abs(to_host(o) - want)) <= 6 * 2.0 ** -8


def test_batch_barrier_timeout_is_reported_and_context_survives(lope):
    """A block that never arrives makes the others' bounded waits run out."""
    shapes, kinds = LI.batch_shapes(83, 4, lo=64, hi=128)
    grids, ins, _ = _batch_setup(lope, shapes, kinds, "f32", 84)
    st = lope.Stencil.builtin("jacobi5", 0.2)
    lope.lope_set_option("wait_limit_ms", 100)
    lope.lope_set_option("batch_skip_arrive", 0)
    try:
        lope.apply_batch(grids, st, ins, nsteps=4, launch=lope.Launch(2, 64, 32, 1, -1))
        with pytest.raises(lope.LopeError, match="TIMEOUT"):
            lope.sync_status()
    finally:
        lope.lope_set_option("batch_skip_arrive", -1)
        lope.lope_set_option("wait_limit_ms", 1000)
    outs = lope.apply_batch(grids, st, ins, nsteps=4, launch=lope.Launch(2, 64, 32, 1, -1))
    lope.sync_status()
    for g, i, o in zip(grids, ins, outs):
        assert torch.equal(lope.apply(g, st, i, nsteps=4, launch=lope.Launch(2, 64, 32, 1, -1)), o)


def test_batch_full_size_512_grids_bitwise_vs_per_grid(lope, orc, error_report):
    """The 512-grid batch: every 37th grid bitwise against its own per-grid run
    and, with the smallest grid, element by element against the oracle within
    T eps (error_bounds.py; the 5-point weights at c = 0.2 are non-negative, so
    the impulse norms are 1)."""
    shapes, kinds = LI.batch_shapes(1003, 512)
    grids, ins, stored = _batch_setup(lope, shapes, kinds, "f32", 1003)
    st = lope.Stencil.builtin("jacobi5", 0.2)
    T = 20
    launch = lope.Launch(2, 64, 32, 4, -1)
    outs = lope.apply_batch(grids, st, ins, nsteps=T, launch=launch)
    torch.cuda.synchronize()
    lope.sync_status()
    small = int(np.argmin([a * b for a, b in shapes]))
    bound = T * float(local_eps("jacobi5", [0.2], [1.0], "f32")[0])
    worst, pts = 0.0, 0
    for gi in sorted(set(range(0, 512, 37)) | {small}):
        alone = lope.apply(grids[gi], st, ins[gi], nsteps=T, launch=launch)
        torch.cuda.synchronize()
        assert torch.equal(alone, outs[gi]), gi
        want = orc.apply(stored[gi], "jacobi5", [0.2], T, bc=[kinds[gi]] * 2,
                         nthreads=orc.max_threads())
        err = float(np.max(np.abs(to_host(outs[gi]) - want)))
        worst, pts = max(worst, err), pts + want.size
        assert err <= bound, (gi, err, bound)
    error_report["K5 batched jacobi5 FP32 512 grids x20 (15 grids, full)"] = {
        "max_abs": worst, "bound": bound, "points": pts}


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("ckpt", [10, 7, 100, 1])
def test_adjoint_fp64_32cube_vs_oracle(lope, orc, ckpt):
    shape, c, T = (32, 32, 32), 0.1, 100
    u0, u0s = to_device(LI.uniform_field(1004, shape), "f64")
    tg, tgs = to_device(LI.normal_field(2004, shape), "f64")
    g = lope.Grid(shape, "f64", halo=1)
    st = lope.Stencil.builtin("diff7", c)
    loss, gu, gc = lope.adjoint(g, st, u0, tg, T, ckpt)
    loss_o, gu_o, gc_o = orc.adjoint(u0s, tgs, "diff7", [c], T, nthreads=orc.max_threads())
    assert abs(loss - loss_o) <= 1e-12 * loss_o
    assert normwise(to_host(gu), gu_o) <= 1e-12
    assert abs(gc - gc_o) <= 1e-12 * abs(gc_o)


def test_adjoint_f32_32cube_vs_oracle_and_fd(lope, orc, error_report):
    shape, c, T, eps = (32, 32, 32), 0.1, 100, 1e-3
    u0, u0s = to_device(LI.uniform_field(1004, shape), "f32")
    tg, tgs = to_device(LI.normal_field(2004, shape), "f32")
    g = lope.Grid(shape, "f32", halo=1)
    st = lope.Stencil.builtin("diff7", c)
    loss, gu, gc = lope.adjoint(g, st, u0, tg, T, 10)
    loss_o, gu_o, gc_o = orc.adjoint(u0s, tgs, "diff7", [c], T, nthreads=orc.max_threads())
    rel = {"loss": abs(loss - loss_o) / loss_o, "dL_du0_normwise": normwise(to_host(gu), gu_o),
           "dL_dc": abs(gc - gc_o) / abs(gc_o)}
    assert rel["loss"] <= 1e-4
    assert rel["dL_du0_normwise"] <= 1e-4
    assert rel["dL_dc"] <= 1e-4

    def L(cc):
        uT = orc.apply(u0s, "diff7", [cc], T, nthreads=orc.max_threads())
        return float(np.sum((uT - tgs) ** 2))

    fd = (L(c + eps) - L(c - eps)) / (2 * eps)
    rel["dL_dc_vs_central_fd"] = abs(fd - gc) / abs(fd)
    assert rel["dL_dc_vs_central_fd"] <= 2e-3
    error_report["K6 adjoint diff7 FP32 32^3 x100, checkpoint 10 (relative)"] = {
        "measured": rel, "bound": {"vs_discrete_adjoint": 1e-4, "vs_central_fd": 2e-3}}


def test_adjoint_2d_stencils_and_dirichlet(lope, orc):
    for kind, c, bc, halo in (("jacobi5", 0.2, [1, 1], 1), ("jacobi5", 0.2, [0, 1], 1),
                              ("star9r2", 0.1, [0, 0], 2), ("star9r2", 0.1, [1, 0], 2)):
        shape, T = (45, 72), 23
        u0, u0s = to_device(LI.uniform_field(90, shape), "f64")
        tg, tgs = to_device(LI.normal_field(91, shape), "f64")
        g = lope.Grid(shape, "f64", halo=halo)
        g.set_boundaries(bc)
        st = lope.Stencil.builtin(kind, c)
        loss, gu, gc = lope.adjoint(g, st, u0, tg, T, 5)
        loss_o, gu_o, gc_o = orc.adjoint(u0s, tgs, kind, [c], T, bc=bc)
        assert abs(loss - loss_o) <= 1e-12 * loss_o, kind
        assert normwise(to_host(gu), gu_o) <= 1e-12, kind
        assert abs(gc - gc_o) <= 1e-11 * abs(gc_o), kind


def test_adjoint_linear_asymmetric_reflects_offsets(lope, orc):
    w = LI.uniform_field(92, (3, 3, 3)) * 0.2 - 0.1
    mask = np.zeros_like(w)
    for ax in range(3):
        for d in range(3):
            idx = [1, 1, 1]
            idx[ax] = d
            mask[tuple(idx)] = 1
    w = w * mask
    shape, T = (9, 10, 24), 6
    for bc in ([0, 0, 0], [1, 0, 1]):
        u0, u0s = to_device(LI.uniform_field(93, shape), "f64")
        lam, lams = to_device(LI.normal_field(94, shape), "f64")
        g = lope.Grid(shape, "f64", halo=1)
        g.set_boundaries(bc)
        st = lope.Stencil.linear(w)
        gu, gc = lope.vjp(g, st, u0, lam, T, 4)
        gu_o, _ = orc.vjp(u0s, lams, "linear", nsteps=T, bc=bc, weights_table=w)
        assert normwise(to_host(gu), gu_o) <= 1e-12
        assert float(gc.item()) == 0.0


def test_autograd_function_matches_oracle(lope, orc):
    from paper_1502_03504_gb300.autograd import DiffusionFn

    shape, T = (16, 20, 24), 30
    u0, u0s = to_device(LI.uniform_field(95, shape), "f64")
    tg, tgs = to_device(LI.normal_field(96, shape), "f64")
    u0.requires_grad_(True)
    coeff = torch.tensor(0.1, dtype=torch.float64, device="cuda", requires_grad=True)
    uT = DiffusionFn.apply(u0, coeff, T, "diff7", None, 7)
    loss = ((uT - tg) ** 2).sum()
    loss.backward()
    loss_o, gu_o, gc_o = orc.adjoint(u0s, tgs, "diff7", [0.1], T)
    assert abs(float(loss) - loss_o) <= 1e-12 * loss_o
    assert normwise(to_host(u0.grad), gu_o) <= 1e-12
    assert abs(float(coeff.grad) - gc_o) <= 1e-12 * abs(gc_o)


def test_adjoint_full_size_256_dot_product(lope):
    """<A^T x, y> = <x, (A^T)^T y> for the 100-step periodic operator at 256^3."""
    shape, c, T = (256, 256, 256), 0.1, 100
    x, _ = to_device(LI.uniform_field(1004, shape), "f32")
    y, _ = to_device(LI.normal_field(2004, shape), "f32")
    g = lope.Grid(shape, "f32", halo=1)
    st = lope.Stencil.builtin("diff7", c)
    Ax = lope.apply(g, st, x, nsteps=T)
    ATy, gc = lope.vjp(g, st, x, y, T, 10)
    torch.cuda.synchronize()
    lope.sync_status()
    lhs = float(torch.sum(Ax.double() * y.double()))
    rhs = float(torch.sum(x.double() * ATy.double()))
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + float(torch.sum(torch.abs(Ax.double() * y.double()))) * 1e-2)
    assert np.isfinite(float(gc.item()))


def test_batch_autotuner_choice_is_used_and_bitwise_equal(lope):
    """lope_autotune_batch stores its choice; a later lope_apply_batch with no
    launch configuration uses it, and gives bitwise what the explicit choice
    (and each grid advanced alone with that tile and depth) gives."""
    shapes = [(70, 130), (33, 257), (128, 64), (200, 201), (5, 300)]
    kinds = [0, 1, 1, 0, 1]
    grids, ins, _ = _batch_setup(lope, shapes, kinds, "f32", 1600)
    st = lope.Stencil.builtin("jacobi5", 0.2)
    outs = [torch.empty_like(x) for x in ins]
    works = [torch.empty_like(x) for x in ins]
    best, ms = lope.autotune_batch(grids, st, ins, outs, works, 9)
    assert best.path == 2 and best.tile_x in (64, 128) and best.tsteps in (1, 2, 4, 5) and ms > 0
    auto = [o.clone() for o in lope.apply_batch(grids, st, ins, nsteps=9)]
    explicit = lope.apply_batch(grids, st, ins, nsteps=9,
                                launch=lope.Launch(2, best.tile_x, best.tile_y, best.tsteps, -1))
    torch.cuda.synchronize()
    lope.sync_status()
    for a, b, g, i in zip(auto, explicit, grids, ins):
        assert torch.equal(a, b)
        alone = lope.apply(g, st, i, nsteps=9,
                           launch=lope.Launch(2, best.tile_x, best.tile_y, best.tsteps, -1))
        torch.cuda.synchronize()
        assert torch.equal(alone, a)


@pytest.mark.parametrize("kind,prm,halo", [("jacobi5", [0.2], 1), ("star9r2", [0.1], 2)])
def test_batch_two_sweep_tiles_equal_per_grid_and_oracle(lope, orc, kind, prm, halo):
    """The two-sweep batched tiles (path 1): uneven grids of any row pitch,
    periodic and Dirichlet sides (non-zero values included), even and odd step
    counts (an odd count ends with a one-sweep pass): bitwise equal to each
    grid advanced alone, and within T eps of the oracle."""
    shapes, kinds = LI.batch_shapes(85, 12, lo=5, hi=400)
    shapes[0], shapes[1] = (1, 7), (130, 3)  # a single row; fewer columns than the radius
    kinds[0], kinds[1] = 1, 1
    bvals = [((0.3, -0.2), (0.0, 0.5)) if k == 1 and i % 2 else ((0.0, 0.0), (0.0, 0.0))
             for i, k in enumerate(kinds)]
    grids, ins, stored = [], [], []
    off = 0
    for (ny, nx), k, bv in zip(shapes, kinds, bvals):
        g = lope.Grid((ny, nx), "f32", halo=halo)
        if k == 1:
            g.set_boundaries([(1, 1), (1, 1)], list(bv))
        grids.append(g)
        u = LI.uniform(86, ny * nx, off).reshape(ny, nx)
        off += ny * nx
        t, st_ = to_device(u, "f32")
        ins.append(t)
        stored.append(st_)
    st = lope.Stencil.builtin(kind, *prm)
    for T in (6, 7):
        outs = lope.apply_batch(grids, st, ins, nsteps=T, launch=lope.Launch(1, 64, 128, 2, -1))
        torch.cuda.synchronize()
        lope.sync_status()
        for gi, (g, i, o) in enumerate(zip(grids, ins, outs)):
            alone = lope.apply(g, st, i, nsteps=T, launch=lope.Launch(3, 0, 0, 0, -1))
            torch.cuda.synchronize()
            assert torch.equal(alone, o), (T, gi, shapes[gi])
    for gi in (0, 1, 2, 5):
        k = kinds[gi]
        bc = [(k, k), (k, k)]
        want = orc.apply(stored[gi], kind, prm, 7, bc=bc, bval=list(bvals[gi]))
        G = 1.0 if kind == "jacobi5" else 1.0667
        M = max(1.0, *(abs(v) for pair in bvals[gi] for v in pair))
        eps = float(local_eps(kind, prm, [M * G ** 7], "f32")[0])
        assert np.max(np.abs(to_host(outs[gi]) - want)) <= 7 * G ** 7 * eps, gi
