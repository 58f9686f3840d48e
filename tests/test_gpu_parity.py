"""GPU parity: the CUDA kernels (through the C ABI) against the FP64 oracle.

Small cases span several tiles and a ragged tail and are compared element by
element; the full-size workloads are compared on sampled outputs, each of
which the oracle computes on the sub-box that can influence it (the domain of
dependence of T steps of a radius-R stencil is R*T cells wide, so cutting the
box further out does not change the sampled value).
"""
import numpy as np
import pytest
import torch

import lope_inputs as LI
from error_bounds import growth, impulse_norms, local_eps, sup_bound
from gpu_helpers import bound_bf16, bound_f32, normwise, sub_box, to_device, to_host

pytestmark = pytest.mark.gpu

TMA, TRAP, DIRECT = 1, 2, 3


def _launch(L, path, tx=0, ty=0, k=0, graph=-1):
    return L.Launch(path, tx, ty, k, graph)


def _grid(L, shape, dtype, halo, bc, bval=None, nf=1):
    g = L.Grid(shape, dtype, halo=halo, nfields=nf)
    g.set_boundaries(bc, bval)
    return g


def _run(L, g, st, fields, nsteps, launch=None):
    out = L.apply(g, st, fields, nsteps=nsteps, launch=launch)
    torch.cuda.synchronize()
    L.sync_status()
    return out


# ------------------------------------------------------------------ K1: FP64, 1e-12
@pytest.mark.parametrize("path", [0, TMA, TRAP, DIRECT])
def test_jacobi5_fp64_256_periodic_100(lope, orc, path, error_report):
    shape, c, T = (256, 256), 0.2, 100
    u0, u0s = to_device(LI.uniform_field(1000, shape), "f64")
    g = _grid(lope, shape, "f64", 1, [0, 0])
    st = lope.Stencil.builtin("jacobi5", c)
    got = to_host(_run(lope, g, st, u0, T, None if path == 0 else _launch(lope, path, k=1)))
    want = orc.apply(u0s, "jacobi5", [c], T)
    rel = normwise(got, want)
    key = "K1 jacobi5 FP64 256^2 x100 (normwise relative, every path)"
    prev = error_report.get(key, {}).get("normwise", 0.0)
    error_report[key] = {"normwise": max(prev, rel), "bound": 1e-12,
                         "max_abs": max(error_report.get(key, {}).get("max_abs", 0.0),
                                        float(np.max(np.abs(got - want))))}
    assert rel <= 1e-12


def test_jacobi5_fp64_all_paths_bitwise(lope):
    shape, c, T = (256, 256), 0.2, 24
    u0, _ = to_device(LI.uniform_field(1000, shape), "f64")
    g = _grid(lope, shape, "f64", 1, [0, 0])
    st = lope.Stencil.builtin("jacobi5", c)
    ref = _run(lope, g, st, u0, T, _launch(lope, TMA))
    for launch in (_launch(lope, DIRECT), _launch(lope, TRAP, 64, 32, 1), _launch(lope, TRAP, 32, 8, 3),
                   _launch(lope, TRAP, 128, 16, 8), _launch(lope, TMA, graph=1)):
        assert torch.equal(_run(lope, g, st, u0, T, launch), ref), launch


# ------------------------------------------------------------------ 2D FP32, ragged tiles
@pytest.mark.parametrize("bc,bval", [([0, 0], None), ([1, 1], None), ([1, 0], [0.0, 0.0]),
                                     ([(1, 1), (1, 1)], [(0.5, -0.25), (1.0, 0.0)])])
@pytest.mark.parametrize("path", [0, TRAP, DIRECT])
def test_jacobi5_f32_ragged(lope, orc, bc, bval, path):
    shape, c, T = (75, 200), 0.2, 17
    u0, u0s = to_device(LI.uniform_field(1, shape), "f32")
    g = _grid(lope, shape, "f32", 1, bc, bval)
    st = lope.Stencil.builtin("jacobi5", c)
    launch = None if path == 0 else _launch(lope, path, 64, 32, 3 if path == TRAP else 1)
    got = to_host(_run(lope, g, st, u0, T, launch))
    want = orc.apply(u0s, "jacobi5", [c], T, bc=bc, bval=bval)
    M = max(1.0, np.max(np.abs(want)), *(abs(v) for v in np.ravel(bval or [0.0])))
    assert np.max(np.abs(got - want)) <= bound_f32(T, M, nops=7)


def test_star9r2_f32_periodic_ragged(lope, orc):
    shape, c, T = (70, 136), 0.1, 12
    u0, u0s = to_device(LI.uniform_field(2, shape), "f32")
    g = _grid(lope, shape, "f32", 2, [0, 0])
    st = lope.Stencil.builtin("star9r2", c)
    want = orc.apply(u0s, "star9r2", [c], T)
    G = abs(1 - 5 * c) + c * (4 * 4 / 3 + 4 / 12)  # ||I + cL||_inf
    for launch in (None, _launch(lope, TRAP, 64, 16, 2), _launch(lope, DIRECT)):
        got = to_host(_run(lope, g, st, u0, T, launch))
        assert np.max(np.abs(got - want)) <= bound_f32(T, 1.0, nops=12, G=G)


def test_star9r2_dirichlet_small_axes(lope, orc):
    """Grids narrower than a tile in both axes; Dirichlet with a non-zero value."""
    shape, c, T = (5, 12), 0.1, 6
    u0, u0s = to_device(LI.uniform_field(3, shape), "f32")
    g = _grid(lope, shape, "f32", 2, [1, 1], [0.3, -0.2])
    st = lope.Stencil.builtin("star9r2", c)
    want = orc.apply(u0s, "star9r2", [c], T, bc=[1, 1], bval=[0.3, -0.2])
    for launch in (None, _launch(lope, TRAP, 32, 8, 4), _launch(lope, DIRECT)):
        got = to_host(_run(lope, g, st, u0, T, launch))
        assert np.max(np.abs(got - want)) <= bound_f32(T, 1.0, nops=12, G=3.0)


# ------------------------------------------------------------------ 3D
@pytest.mark.parametrize("bc", [[1, 1, 1], [0, 0, 0], [0, 1, 0], [1, 0, 1]])
def test_diff7_f32_ragged(lope, orc, bc):
    shape, c, T = (37, 50, 72), 0.1, 12
    u0, u0s = to_device(LI.uniform_field(4, shape), "f32")
    g = _grid(lope, shape, "f32", 1, bc)
    st = lope.Stencil.builtin("diff7", c)
    want = orc.apply(u0s, "diff7", [c], T, bc=bc)
    ref = None
    for launch in (None, _launch(lope, TMA), _launch(lope, DIRECT)):
        out = _run(lope, g, st, u0, T, launch)
        got = to_host(out)
        assert np.max(np.abs(got - want)) <= bound_f32(T, 1.0, nops=9), launch
        if ref is None:
            ref = out
        else:
            assert torch.equal(out, ref), "TMA and direct paths differ bitwise"


def test_diff7_fp64_periodic_1e12(lope, orc):
    shape, c, T = (20, 33, 48), 0.1, 15
    u0, u0s = to_device(LI.uniform_field(5, shape), "f64")
    g = _grid(lope, shape, "f64", 1, [0, 0, 0])
    st = lope.Stencil.builtin("diff7", c)
    got = to_host(_run(lope, g, st, u0, T))
    assert normwise(got, orc.apply(u0s, "diff7", [c], T)) <= 1e-12


def test_diff7_nz_smaller_than_chunk_and_thin_grids(lope, orc):
    for shape, bc in (((1, 8, 8), [0, 0, 0]), ((3, 4, 128), [1, 0, 0]), ((64, 2, 4), [0, 1, 0])):
        u0, u0s = to_device(LI.uniform_field(6, shape), "f32")
        g = _grid(lope, shape, "f32", 1, bc)
        st = lope.Stencil.builtin("diff7", 0.1)
        got = to_host(_run(lope, g, st, u0, 5))
        want = orc.apply(u0s, "diff7", [0.1], 5, bc=bc)
        assert np.max(np.abs(got - want)) <= bound_f32(5, 1.0, nops=9), shape


# ------------------------------------------------------------------ linear stencils
@pytest.mark.parametrize("ndim,r,box", [(2, 1, False), (2, 2, False), (3, 1, False), (2, 1, True),
                                        (2, 2, True), (3, 1, True)])
def test_linear_asymmetric_fp64(lope, orc, ndim, r, box):
    side = 2 * r + 1
    w = LI.uniform_field(50 + ndim * 10 + r, (side,) * ndim) * 0.2 - 0.1
    if not box:  # keep axis taps only
        mask = np.zeros_like(w)
        ctr = (r,) * ndim
        for ax in range(ndim):
            for d in range(side):
                idx = list(ctr)
                idx[ax] = d
                mask[tuple(idx)] = 1
        w = w * mask
    shape = (41, 68) if ndim == 2 else (9, 13, 36)
    bc = [0] * ndim if r == 1 else [1] * ndim
    u0, u0s = to_device(LI.uniform_field(7, shape), "f64")
    g = _grid(lope, shape, "f64", r, bc)
    st = lope.Stencil.linear(w)
    got = to_host(_run(lope, g, st, u0, 4))
    want = orc.apply(u0s, "linear", nsteps=4, bc=bc, weights_table=w)
    assert normwise(got, want) <= 1e-12


# ------------------------------------------------------------------ multi-field
def test_swe_f32_and_bf16(lope, orc, error_report):
    """Small linear shallow-water runs on every path against the derived
    sup-norm and mean bounds (see test_full_size_swe_4096_200_sampled)."""
    shape, T = (40, 72), 20
    prm = [0.02, 1.0, 1.0]
    h, u, v = LI.swe_fields(1002, shape)
    st = lope.Stencil.builtin("swe_cgrid", *prm)
    norms = impulse_norms(orc, "swe_cgrid", prm, 3, 2, 1, T)
    # FP32 stores h; BF16 stores eta = h - H (perturbation storage)
    for dtype, first in (("f32", h), ("bf16", h - 1.0)):
        dev, stored = zip(*(to_device(f, dtype) for f in (first, u, v)))
        g = _grid(lope, shape, dtype, 1, [0, 0], nf=3)
        _, M, D = _stepwise_swe(lope, g, st, dev, T)
        eps = local_eps("swe_cgrid", prm, M, dtype, dh=D)
        sup = sup_bound(norms, eps)
        want = orc.apply(list(stored), "swe_cgrid", prm, T)
        worst = [0.0] * 3
        for launch in (None, _launch(lope, TRAP, 64, 32, 2), _launch(lope, DIRECT)):
            outs = _run(lope, g, st, list(dev), T, launch)
            for k in range(3):
                got = to_host(outs[k])
                err = float(np.max(np.abs(got - want[k])))
                worst[k] = max(worst[k], err)
                assert err <= sup[k], (dtype, k, launch, err, sup[k])
                assert abs(np.mean(got) - np.mean(stored[k])) <= T * eps[k], (dtype, k, launch)
        error_report[f"K4 swe_cgrid {dtype.upper()} 40x72 x20 (every path)"] = {
            "max_abs": worst, "bound": list(map(float, sup))}


# ------------------------------------------------------------------ edge cases
def test_nsteps_zero_and_one(lope, orc):
    shape = (9, 40)
    u0, u0s = to_device(LI.uniform_field(8, shape), "f32")
    g = _grid(lope, shape, "f32", 1, [0, 0])
    st = lope.Stencil.builtin("jacobi5", 0.2)
    out = torch.empty_like(u0)
    lope.apply(g, st, u0, out=out, nsteps=0)
    torch.cuda.synchronize()
    assert torch.equal(out, u0)
    lope.apply(g, st, u0, out=out, work=None, nsteps=1)
    torch.cuda.synchronize()
    assert np.max(np.abs(to_host(out) - orc.apply(u0s, "jacobi5", [0.2], 1))) < 1e-6


def test_degenerate_single_row_and_column(lope, orc):
    st = lope.Stencil.builtin("jacobi5", 0.2)
    for shape in ((1, 7), (7, 1), (1, 1)):
        u0, u0s = to_device(LI.uniform_field(9, shape), "f32")
        g = _grid(lope, shape, "f32", 1, [0, 0])
        got = to_host(_run(lope, g, st, u0, 3))
        assert np.max(np.abs(got - orc.apply(u0s, "jacobi5", [0.2], 3))) < 1e-6, shape


def test_input_is_never_written_and_aliasing_rejected(lope):
    shape = (64, 64)
    u0, _ = to_device(LI.uniform_field(10, shape), "f32")
    keep = u0.clone()
    g = _grid(lope, shape, "f32", 1, [0, 0])
    st = lope.Stencil.builtin("jacobi5", 0.2)
    _run(lope, g, st, u0, 7)
    assert torch.equal(u0, keep)
    with pytest.raises(lope.LopeError, match="alias"):
        lope.apply(g, st, u0, out=u0, nsteps=1)
    with pytest.raises(lope.LopeError, match="aligned"):
        lope.apply(g, st, u0, out=torch.empty(64 * 64 + 1, device="cuda")[1:].view(64, 64), nsteps=1)


def test_launch_counter_counts_kernels(lope):
    shape = (64, 64)
    u0, _ = to_device(LI.uniform_field(11, shape), "f32")
    g = _grid(lope, shape, "f32", 1, [0, 0])
    st = lope.Stencil.builtin("jacobi5", 0.2)
    before = lope.launch_count()
    _run(lope, g, st, u0, 5, _launch(lope, TMA))
    assert lope.launch_count() - before == 5
    before = lope.launch_count()
    _run(lope, g, st, u0, 8, _launch(lope, TRAP, 64, 32, 4))
    assert lope.launch_count() - before == 2


# ------------------------------------------------------------------ reductions
def test_fp64_reductions(lope):
    x64 = LI.uniform_field(12, (1000, 777))
    y64 = LI.normal_field(13, (1000, 777))
    for dtype in ("f32", "bf16", "f64"):
        x, xs = to_device(x64, dtype)
        y, ys = to_device(y64, dtype)
        s = float(lope.reduce_sum(x).item())
        q = float(lope.reduce_sqdiff(x, y).item())
        assert abs(s - xs.sum()) <= 1e-9 * abs(xs.sum())
        assert abs(q - np.sum((xs - ys) ** 2)) <= 1e-9 * q


def test_sum_conserved_periodic_on_gpu(lope):
    shape = (96, 160)
    u0, _ = to_device(LI.uniform_field(14, shape), "f64")
    g = _grid(lope, shape, "f64", 1, [0, 0])
    st = lope.Stencil.builtin("jacobi5", 0.2)
    out = _run(lope, g, st, u0, 50)
    a = float(lope.reduce_sum(u0).item())
    b = float(lope.reduce_sum(out).item())
    assert abs(a - b) <= 1e-12 * abs(a)


# ------------------------------------------------------------------ full-size, sampled
def _sampled_check(lope, orc, kind, prm, shape, bc, T, R, dtype, nf_fields, got_fields, stored,
                   points, tol_fn):
    """Compare sampled outputs with the oracle on their domains of dependence;
    returns the largest error seen per field."""
    periodic = [b == 0 for b in bc]
    rho = R * T + 1
    worst = [0.0] * nf_fields
    for p in points:
        idx, pos = sub_box(shape, p, rho, periodic)
        sub = [s[np.ix_(*idx)] for s in stored]
        sub_bc = []
        for ax, n in enumerate(shape):
            full = len(idx[ax]) == n and (not periodic[ax] or 2 * rho + 1 >= n)
            sub_bc.append(0 if (periodic[ax] and full) else 1)
        want = orc.apply(sub if nf_fields > 1 else sub[0], kind, prm, T, bc=sub_bc,
                         nthreads=orc.max_threads())
        want = want if nf_fields > 1 else [want]
        for k in range(nf_fields):
            w = want[k][pos]
            gv = float(got_fields[k][p].item())
            worst[k] = max(worst[k], abs(gv - w))
            assert abs(gv - w) <= tol_fn(k, w), (p, k, gv, w)
    return worst


def _scalar_bound(orc, kind, prm, ndim, R, T, M):
    """Sup-norm bound of an FP32 run of a one-field builtin (error_bounds.py):
    the local error of one step, from the operation tree, carried by the
    impulse-response norms of the exact steps."""
    norms = impulse_norms(orc, kind, prm, 1, ndim, R, T)
    return float(sup_bound(norms, local_eps(kind, prm, [growth(norms) * M], "f32"))[0])


def test_full_size_diff7_512_dirichlet_50_sampled(lope, orc, error_report):
    shape, c, T = (512, 512, 512), 0.1, 50
    u0, u0s = to_device(LI.uniform_field(1001, shape), "f32")
    g = _grid(lope, shape, "f32", 1, [1, 1, 1])
    st = lope.Stencil.builtin("diff7", c)
    out = _run(lope, g, st, u0, T)
    bound = _scalar_bound(orc, "diff7", [c], 3, 1, T, np.max(np.abs(u0s)))
    pts = [(0, 0, 0), (511, 511, 511), (0, 255, 511), (256, 256, 256), (100, 3, 400), (511, 0, 7)]
    worst = _sampled_check(lope, orc, "diff7", [c], shape, [1, 1, 1], T, 1, "f32", 1, [out], [u0s],
                           pts, lambda k, w: bound)
    error_report["K2 diff7 FP32 512^3 x50 (sampled)"] = {"max_abs": worst[0], "bound": bound}


def test_full_size_star9r2_8192_periodic_50_sampled(lope, orc, error_report):
    shape, c, T = (8192, 8192), 0.1, 50
    u0, u0s = to_device(LI.uniform_field(1001, shape, offset=1 << 32), "f32")
    g = _grid(lope, shape, "f32", 2, [0, 0])
    st = lope.Stencil.builtin("star9r2", c)
    out = _run(lope, g, st, u0, T)
    bound = _scalar_bound(orc, "star9r2", [c], 2, 2, T, np.max(np.abs(u0s)))
    pts = [(0, 0), (8191, 8191), (0, 4096), (4000, 8191), (1234, 5678), (8190, 1)]
    worst = _sampled_check(lope, orc, "star9r2", [c], shape, [0, 0], T, 2, "f32", 1, [out], [u0s],
                           pts, lambda k, w: bound)
    error_report["K3 star9r2 FP32 8192^2 x50 (sampled)"] = {"max_abs": worst[0], "bound": bound}


def _full_field(lope, orc, kind, c, shape, bc, T, R, seed_args, error_report, key):
    """The complete output of a headline workload against the oracle, element by
    element (the oracle on every host core)."""
    u0, u0s = to_device(LI.uniform_field(*seed_args), "f32")
    g = _grid(lope, shape, "f32", R, bc)
    st = lope.Stencil.builtin(kind, c)
    out = to_host(_run(lope, g, st, u0, T))
    del u0
    want = orc.apply(u0s, kind, [c], T, bc=bc, nthreads=orc.max_threads())
    err = float(np.max(np.abs(out - want)))
    bound = _scalar_bound(orc, kind, [c], len(shape), R, T, np.max(np.abs(u0s)))
    error_report[key] = {"max_abs": err, "bound": bound, "points": int(out.size)}
    assert err <= bound, (err, bound)


def test_full_field_diff7_512_dirichlet_50(lope, orc, error_report):
    _full_field(lope, orc, "diff7", 0.1, (512, 512, 512), [1, 1, 1], 50, 1,
                (1001, (512, 512, 512)), error_report, "K2 diff7 FP32 512^3 x50 (full field)")


def test_full_field_star9r2_8192_periodic_50(lope, orc, error_report):
    _full_field(lope, orc, "star9r2", 0.1, (8192, 8192), [0, 0], 50, 2,
                (1001, (8192, 8192), 1 << 32), error_report,
                "K3 star9r2 FP32 8192^2 x50 (full field)")


def _stepwise_swe(lope, g, st, dev, T):
    """The run one step at a time (bitwise the same as one call of T steps);
    returns the final state, the largest magnitude of each field over all
    states, and the largest neighbour difference of field 0 (the magnitudes the
    local error bound of every step depends on)."""
    cur = list(dev)
    M = [float(x.float().abs().max()) for x in cur]

    def maxdiff(x):
        x = x.float()
        return max(float((torch.roll(x, -1, d) - x).abs().max()) for d in (0, 1))

    D = maxdiff(cur[0])
    for _ in range(T):
        cur = lope.apply(g, st, cur, nsteps=1)
        M = [max(m, float(x.float().abs().max())) for m, x in zip(M, cur)]
        D = max(D, maxdiff(cur[0]))
    torch.cuda.synchronize()
    return cur, M, D


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_full_size_swe_4096_200_sampled(lope, orc, dtype, error_report):
    """Linear C-grid shallow water at 4096^2 x 3 fields, 200 steps, periodic.
    Sup-norm bound: the local error of one step (from the operation tree and
    the magnitudes of the run's own states) carried by the impulse-response
    norms of 200 exact steps (FP32 about 1e-4; BF16 storage has no useful
    worst case at this length).  Mean bound: every field's mean is conserved
    by the exact step, so the mean drifts by at most T eps per field, which a
    bias of one ulp per step exceeds (FP32 and BF16)."""
    shape, T = (4096, 4096), 200
    prm = [0.02, 1.0, 1.0]
    h, u, v = LI.swe_fields(1002, shape)
    first = h if dtype == "f32" else h - 1.0
    dev, stored = zip(*(to_device(f, dtype) for f in (first, u, v)))
    g = _grid(lope, shape, dtype, 1, [0, 0], nf=3)
    st = lope.Stencil.builtin("swe_cgrid", *prm)
    outs = _run(lope, g, st, list(dev), T)
    steps, M, D = _stepwise_swe(lope, g, st, dev, T)
    for k in range(3):
        assert torch.equal(steps[k], outs[k]), k
    norms = impulse_norms(orc, "swe_cgrid", prm, 3, 2, 1, T)
    eps = local_eps("swe_cgrid", prm, M, dtype, dh=D)
    sup = sup_bound(norms, eps)
    pts = [(0, 0), (4095, 4095), (2048, 17), (9, 3000)]
    worst = _sampled_check(lope, orc, "swe_cgrid", prm, shape, [0, 0], T, 1, dtype, 3, outs,
                           list(stored), pts, lambda k, w: sup[k])
    drift = []
    for k in range(3):
        m0 = float(np.mean(stored[k]))
        m1 = float(lope.reduce_sum(outs[k]).item()) / outs[k].numel()
        drift.append(abs(m1 - m0))
        assert drift[k] <= T * eps[k], (k, drift[k], T * eps[k])
    error_report[f"K4 swe_cgrid {dtype.upper()} 4096^2 x200 (sampled)"] = {
        "max_abs": worst, "bound": list(map(float, sup)), "mean_drift": drift,
        "mean_bound": list(map(float, T * eps))}


# ------------------------------------------------------------------ planner / autotuner
def test_autotune_choice_is_bitwise_equal(lope):
    shape = (300, 512)
    u0, _ = to_device(LI.uniform_field(15, shape), "f32")
    g = _grid(lope, shape, "f32", 1, [0, 0])
    st = lope.Stencil.builtin("jacobi5", 0.2)
    ref = _run(lope, g, st, u0, 12, _launch(lope, TMA))
    out, work = torch.empty_like(u0), torch.empty_like(u0)
    best, ms = lope.autotune(g, st, u0, out, work, 12)
    assert best.path in (TMA, TRAP, DIRECT) and ms > 0
    # the remembered choice is what lope_apply now uses; any choice is bitwise equal
    assert torch.equal(_run(lope, g, st, u0, 12), ref)


def test_bf16_tma_jacobi5_vs_oracle(lope, orc):
    shape, c, T = (96, 128), 0.2, 10
    u0, u0s = to_device(LI.uniform_field(16, shape), "bf16")
    g = _grid(lope, shape, "bf16", 1, [0, 1])
    st = lope.Stencil.builtin("jacobi5", c)
    want = orc.apply(u0s, "jacobi5", [c], T, bc=[0, 1])
    for launch in (_launch(lope, TMA), _launch(lope, TRAP, 64, 16, 3), _launch(lope, DIRECT)):
        got = to_host(_run(lope, g, st, u0, T, launch))
        assert np.max(np.abs(got - want)) <= bound_bf16(T, 1.0, 7), launch


def test_graph_replay_matches_direct_launches(lope):
    shape = (256, 256)
    u0, _ = to_device(LI.uniform_field(17, shape), "f32")
    g = _grid(lope, shape, "f32", 1, [1, 1])
    st = lope.Stencil.builtin("jacobi5", 0.2)
    direct = _run(lope, g, st, u0, 40, _launch(lope, TMA, graph=-1))
    out, work = torch.empty_like(u0), torch.empty_like(u0)
    for _ in range(3):  # capture once, replay twice
        lope.apply(g, st, u0, out=out, work=work, nsteps=40, launch=_launch(lope, TMA, graph=1))
    torch.cuda.synchronize()
    assert torch.equal(out, direct)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("kind,halo,prm,nf", [("jacobi5", 1, [0.2], 1), ("star9r2", 2, [0.1], 1),
                                              ("swe_cgrid", 1, [0.02, 1.0, 1.0], 3)])
@pytest.mark.parametrize("bc", [[0, 0], [1, 1], [0, 1]])
def test_2d_paths_bitwise_equal(lope, dtype, kind, halo, prm, nf, bc):
    """Paired TMA columns, the trapezoid tiles and the direct kernel evaluate the
    same rounded operations: results are bitwise equal, ragged tiles included."""
    shape = (70, 136)
    fields = [to_device(LI.uniform_field(60 + k, shape), dtype)[0] for k in range(nf)]
    g = _grid(lope, shape, dtype, halo, bc, nf=nf)
    st = lope.Stencil.builtin(kind, *prm)
    ref = _run(lope, g, st, fields if nf > 1 else fields[0], 9, _launch(lope, DIRECT))
    for launch in (_launch(lope, TMA), _launch(lope, TRAP, 64, 16, 3)):
        got = _run(lope, g, st, fields if nf > 1 else fields[0], 9, launch)
        for a, b in zip(got if nf > 1 else [got], ref if nf > 1 else [ref]):
            assert torch.equal(a, b), (launch, dtype, kind, bc)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("stencil", ["diff7", "star_r1", "star_r2"])
@pytest.mark.parametrize("bc", [[0, 0, 0], [1, 1, 1], [1, 0, 1]])
def test_3d_paths_bitwise_equal(lope, dtype, stencil, bc):
    """The TMA z-march (paired columns for FP32/BF16 storage) and the direct
    kernel evaluate the same rounded operations: results are bitwise equal on
    a grid with ragged tiles in x and y."""
    shape = (21, 40, 136)
    if stencil == "diff7":
        st, halo = lope.Stencil.builtin("diff7", 0.1), 1
    else:
        r = 2 if stencil == "star_r2" else 1
        w = np.asarray(LI.uniform_field(70 + r, (2 * r + 1,) * 3), dtype=np.float64) * 0.05
        mask = np.zeros_like(w, dtype=bool)
        mask[r, r, :] = mask[r, :, r] = mask[:, r, r] = True
        w = np.where(mask, w, 0.0)
        st, halo = lope.Stencil.linear(w), r
    u0, _ = to_device(LI.uniform_field(64, shape), dtype)
    g = _grid(lope, shape, dtype, halo, bc)
    ref = _run(lope, g, st, u0, 7, _launch(lope, DIRECT))
    got = _run(lope, g, st, u0, 7, _launch(lope, TMA))
    assert torch.equal(got, ref), (dtype, stencil, bc)
