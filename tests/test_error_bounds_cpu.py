"""The FP32 / BF16 error bounds of the GPU parity tests (error_bounds.py) hold
for a legitimate reduced-precision run and fail for a planted mistake.

The "runs" here are test doubles on the CPU: the FP64 oracle's step rounded to
the storage format after every step (local error up to half an ulp, the
largest a correct storage rounding commits), and the same with a planted bias
of a stated number of ulps per step.  No GPU is involved."""
import numpy as np
import pytest

import lope_inputs as LI
from error_bounds import (gray_scott_majorant, half_ulp, impulse_norms, local_eps,
                          sup_bound)
from user_bodies import GRAY_SCOTT, GRAY_SCOTT_PRM


def _ulp(m, dtype):
    return 2 * half_ulp(m, dtype)


def _double(orc, kind, prm, x0, T, dtype, bias=None, bc=None):
    """T steps of the oracle, each rounded to `dtype` then shifted by bias[f];
    returns the final state, per field the largest magnitude over the run's
    states, and the largest neighbour difference of field 0 (what the local
    error bound of each step depends on)."""
    x = [np.asarray(a, np.float64) for a in x0]
    M = [np.max(np.abs(a)) for a in x]
    D = _maxdiff(x[0])
    for _ in range(T):
        y = orc.apply(x if len(x) > 1 else x[0], kind, prm, 1, bc=bc, nthreads=orc.max_threads())
        y = y if len(x) > 1 else [y]
        x = [np.asarray(LI.to_storage(a, dtype), np.float64) for a in y]
        if bias is not None:
            x = [a + b for a, b in zip(x, bias)]
        M = [max(m, np.max(np.abs(a))) for m, a in zip(M, x)]
        D = max(D, _maxdiff(x[0]))
    return x, M, D


def _maxdiff(a):
    """Largest difference of neighbours along the two fastest axes (periodic)."""
    return max(np.max(np.abs(np.roll(a, -1, ax) - a)) for ax in (-1, -2))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_swe_bounds_hold_for_rounding_and_catch_one_ulp_bias(orc, dtype):
    shape, T, prm = (48, 64), 200, [0.02, 1.0, 1.0]
    h, u, v = LI.swe_fields(1002, shape)
    first = h if dtype == "f32" else h - 1.0
    x0 = [np.asarray(LI.to_storage(f, dtype), np.float64) for f in (first, u, v)]
    y = orc.apply(x0, "swe_cgrid", prm, T, nthreads=orc.max_threads())
    norms = impulse_norms(orc, "swe_cgrid", prm, 3, 2, 1, T)
    good, M, D = _double(orc, "swe_cgrid", prm, x0, T, dtype)
    eps = local_eps("swe_cgrid", prm, M, dtype, dh=D)
    sup = sup_bound(norms, eps)
    mean_bound = T * eps
    for f in range(3):
        assert np.max(np.abs(good[f] - y[f])) <= sup[f]
        assert abs(np.mean(good[f]) - np.mean(x0[f])) <= mean_bound[f]
    # one ulp (of the field's largest magnitude over the run) per step: the mean
    # drifts by T ulps, beyond T eps (eps is below one ulp for these updates,
    # whose last operation is one FMA or one rounding to storage)
    bias = [_ulp(m, dtype) for m in M]
    assert all(e < b for e, b in zip(eps, bias)), (eps, bias)
    bad, _, _ = _double(orc, "swe_cgrid", prm, x0, T, dtype, bias)
    for f in range(3):
        assert abs(np.mean(bad[f]) - np.mean(x0[f])) > mean_bound[f], f
    if dtype == "f32":
        # the sup-norm bound resolves a uniform bias of k ulps per step
        k = int(np.ceil(max(sup[f] / (T * bias[f]) for f in range(3)))) + 1
        assert k <= 15, k
        bad, _, _ = _double(orc, "swe_cgrid", prm, x0, T, dtype, [k * b for b in bias])
        assert all(np.max(np.abs(bad[f] - y[f])) > sup[f] for f in range(3))


@pytest.mark.parametrize("kind,prm,shape,bc,T,kmax", [
    ("diff7", [0.1], (112, 112, 112), [1, 1, 1], 50, 7),
    ("star9r2", [0.1], (96, 128), [0, 0], 50, 8),
])
def test_scalar_bounds_hold_for_rounding_and_catch_a_few_ulps(orc, kind, prm, shape, bc, T, kmax):
    x0 = LI.to_storage(LI.uniform_field(1001, shape), "f32").astype(np.float64)
    ndim, R = len(shape), 2 if kind == "star9r2" else 1
    norms = impulse_norms(orc, kind, prm, 1, ndim, R, T)
    y = orc.apply(x0, kind, prm, T, bc=bc, nthreads=orc.max_threads())
    good, M, _ = _double(orc, kind, prm, [x0], T, "f32", bc=bc)
    sup = float(sup_bound(norms, local_eps(kind, prm, M, "f32"))[0])
    assert np.max(np.abs(good[0] - y)) <= sup
    # a uniform bias of k ulps of the values' magnitude per step reaches T k ulps
    # at points further than R T from every Dirichlet side
    ulp = _ulp(np.max(np.abs(x0)), "f32")
    k = int(np.ceil(sup / (T * ulp))) + 1
    assert k <= kmax, k
    bad, _, _ = _double(orc, kind, prm, [x0], T, "f32", [k * ulp], bc=bc)
    assert np.max(np.abs(bad[0] - y)) > sup


def test_gray_scott_majorant_holds_for_rounding_and_catches_a_bias(orc):
    """Gray-Scott at dt = 1 amplifies perturbations by up to about 1.4 per step
    where u v is large (the autocatalytic term), so the rigorous elementwise
    bound stays below 1e-3 but resolves only a bias of 16 ulps per step (of
    opposite signs on u and v); a correct rounding uses well under 1 % of it."""
    shape, T = (40, 56), 20
    u0 = 1.0 - 0.3 * LI.uniform(1204, shape[0] * shape[1], 0).reshape(shape)
    v0 = 0.25 * LI.uniform(1204, shape[0] * shape[1], shape[0] * shape[1]).reshape(shape)
    x0 = [LI.to_storage(a, "f32").astype(np.float64) for a in (u0, v0)]
    B, y = gray_scott_majorant(orc, GRAY_SCOTT, GRAY_SCOTT_PRM, x0, T)
    assert max(np.max(b) for b in B) < 1e-3

    def run(bias):
        x = [a.copy() for a in x0]
        for _ in range(T):
            x = orc.apply_source(x, GRAY_SCOTT, GRAY_SCOTT_PRM, 1)
            x = [LI.to_storage(a, "f32").astype(np.float64) + b for a, b in zip(x, bias)]
        return x

    good = run([0.0, 0.0])
    for f in range(2):
        assert np.all(np.abs(good[f] - y[f]) <= B[f]), f
    ulp = [_ulp(np.max(np.abs(a)), "f32") for a in x0]
    bad = run([16 * ulp[0], -16 * ulp[1]])
    assert any(np.any(np.abs(bad[f] - y[f]) > B[f]) for f in range(2))
