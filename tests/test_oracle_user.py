"""Pins of the oracle's path for user-written local functions (source text
compiled for the host in FP64): bodies spelling the builtins reproduce the
pinned builtin oracle to rounding, and the Gray-Scott body matches closed forms of its
spatially uniform and linearised behaviour."""
import numpy as np
import pytest

import lope_inputs as LI
from dense_ref import normwise
from user_bodies import DIFF7, GRAY_SCOTT, GRAY_SCOTT_PRM, JACOBI5, STAR_R2_3D, SWE_FLUX


@pytest.mark.parametrize("scheme", ["euler", "rk3"])
@pytest.mark.parametrize("bc,bval", [([0, 0], None), ([1, 1], [0.3, -0.7])])
def test_user_jacobi5_reproduces_builtin(orc, scheme, bc, bval):
    # the body sums neighbours pairwise, the builtin left to right: rounding-level
    u0 = LI.uniform_field(40, (13, 17))
    a = orc.apply(u0, "jacobi5", [0.2], 9, bc=bc, bval=bval, scheme=scheme)
    b = orc.apply_source(u0, JACOBI5, [0.2], 9, bc=bc, bval=bval, scheme=scheme)
    assert normwise(b, a) <= 1e-14


def test_user_diff7_reproduces_builtin(orc):
    u0 = LI.uniform_field(41, (6, 7, 9))
    a = orc.apply(u0, "diff7", [0.1], 5, bc=[1, 0, 1])
    b = orc.apply_source(u0, DIFF7, [0.1], 5, bc=[1, 0, 1])
    assert normwise(b, a) <= 1e-15


def test_user_swe_flux_reproduces_builtin(orc):
    h, u, v = LI.swe_fields(42, (12, 14))
    prm = [0.02, 1.0, 0.5, 1.0]
    a = orc.apply([h - 1, u, v], "swe_flux", prm, 20)
    b = orc.apply_source([h - 1, u, v], SWE_FLUX, prm, 20)
    for k in range(3):
        assert normwise(b[k], a[k]) <= 1e-13


def _padded(u, R, bc, bval):
    """u with an R-wide halo on every side: the wrapped cells for a periodic
    side, the side's constant for a Dirichlet side (star functions read no
    corner, so the order of the axes does not matter)."""
    p = u
    for ax in range(u.ndim):
        if bc[ax] == 0:
            p = np.concatenate([np.take(p, range(-R, 0), axis=ax), p,
                                np.take(p, range(0, R), axis=ax)], axis=ax)
        else:
            lo, hi = bval[ax]
            shape = list(p.shape)
            shape[ax] = R
            p = np.concatenate([np.full(shape, lo), p, np.full(shape, hi)], axis=ax)
    return p


@pytest.mark.parametrize("bc", [[1, 0, 0], [0, 1, 1], [0, 0, 0]])
def test_user_radius_two_3d_matches_brute_force(orc, bc):
    """An asymmetric radius-2 star body in 3D, per-side Dirichlet values: the
    oracle's user path against slices of an explicitly padded array."""
    shape, T, R, (a, b) = (7, 9, 11), 4, 2, (0.03, 0.05)
    bval = [(0.5, -0.3), (-0.25, 0.4), (1.0, 0.2)]
    u = LI.uniform_field(43, shape)
    want = u.copy()
    nz, ny, nx = shape
    for _ in range(T):
        p = _padded(want, R, bc, bval)
        tap = lambda dx, dy, dz: p[R + dz:R + dz + nz, R + dy:R + dy + ny, R + dx:R + dx + nx]
        c = tap(0, 0, 0)
        far = (tap(2, 0, 0) + tap(-2, 0, 0)) + (tap(0, 2, 0) + tap(0, 0, -2))
        near = (tap(1, 0, 0) + tap(0, -1, 0)) + tap(0, 0, 1)
        want = a * (far - 4 * c) + (b * (near - 3 * c) + c)
    got = orc.apply_source(u, STAR_R2_3D, [a, b], T, bc=bc, bval=bval)
    assert normwise(got, want) <= 1e-14


def test_gray_scott_uniform_state_is_the_reaction_map(orc):
    dt, Du, Dv, F, k = GRAY_SCOTT_PRM
    u, v = 0.7, 0.21
    T = 30
    got = orc.apply_source([np.full((5, 6), u), np.full((5, 6), v)], GRAY_SCOTT, GRAY_SCOTT_PRM, T)
    for _ in range(T):  # the reaction terms alone (every Laplacian vanishes)
        u, v = u + dt * (-u * v * v + F * (1 - u)), v + dt * (u * v * v - (F + k) * v)
    assert abs(got[0][2, 3] - u) <= 1e-14 and abs(got[1][4, 1] - v) <= 1e-14
    assert np.ptp(got[0]) == 0 and np.ptp(got[1]) == 0


def test_gray_scott_linearisation_about_the_trivial_state(orc):
    """About (u, v) = (1, 0) the map is linear to first order in the
    perturbation: each Fourier mode decays by 1 + dt(-4D s - F) for u and
    1 + dt(-4D s - F - k) for v, s = sin^2(pi p/N) + sin^2(pi q/N)."""
    dt, Du, Dv, F, k = GRAY_SCOTT_PRM
    n, T, eps = 16, 10, 1e-7
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    p, q = 3, 5
    mode = np.cos(2 * np.pi * (p * i + q * j) / n)
    s = np.sin(np.pi * p / n) ** 2 + np.sin(np.pi * q / n) ** 2
    gu = 1 + dt * (-4 * Du * s - F)
    gv = 1 + dt * (-4 * Dv * s - F - k)
    got = orc.apply_source([1 + eps * mode, eps * mode], GRAY_SCOTT, GRAY_SCOTT_PRM, T)
    assert np.max(np.abs((got[0] - 1) / eps - gu ** T * mode)) <= 1e-5
    assert np.max(np.abs(got[1] / eps - gv ** T * mode)) <= 1e-5
