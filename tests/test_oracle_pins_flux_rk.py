"""Pins of the oracle's nonlinear shallow-water function and its Runge-Kutta
schemes against facts that do not come from the oracle.

swe_flux (eta, u, v on a C-grid; see oracle/lope_oracle.c) is non-linear, so
no dense matrix describes it.  It is pinned by:
  * a uniform state, where every difference vanishes and the update is the
    exact Coriolis rotation (pins the Coriolis sign and averaging weights);
  * exact mass conservation (flux form, periodic);
  * the exact one-step linearisation about a uniform flow (central difference
    of a quadratic map), compared with the Fourier symbol matrix derived by
    hand (pins every shift of the linear part, including both corner taps);
  * separable special cases whose quadratic terms have closed forms from trig
    identities (pin the products and the averaging stencils of the nonlinear
    terms).
The schemes "rk2"/"rk3" are pinned by their stability polynomials
1 + z + z^2/2 (+ z^3/6) on Fourier and Dirichlet sine eigenmodes, by the same
polynomials of the rotation matrix on uniform states, by conservation, and by
brute-force dense matrices of a box stencil with corners.
"""
import numpy as np
import pytest

import lope_inputs as LI
from dense_ref import assemble, normwise, taps

PRM = [0.02, 1.0, 0.5, 1.0]  # dt, g, f, H


def _grid(shape):
    j, i = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    return j.astype(np.float64), i.astype(np.float64)


# ---------------------------------------------------------------- swe_flux
def test_swe_flux_uniform_state_is_coriolis_rotation(orc):
    dt, g, f, H = PRM
    shape, T = (7, 9), 25
    eta0, U0, V0 = 0.3, 0.7, -0.4
    e, u, v = orc.apply([np.full(shape, eta0), np.full(shape, U0), np.full(shape, V0)],
                        "swe_flux", PRM, T)
    M = np.array([[1.0, dt * f], [-dt * f, 1.0]])
    want = np.linalg.matrix_power(M, T) @ np.array([U0, V0])
    assert np.max(np.abs(e - eta0)) <= 1e-15
    assert np.max(np.abs(u - want[0])) <= 1e-14
    assert np.max(np.abs(v - want[1])) <= 1e-14


def test_swe_flux_conserves_mass(orc):
    shape = (24, 20)
    e0 = 0.1 * LI.normal_field(71, shape)
    u0 = 0.2 * LI.normal_field(71, shape, 1000)
    v0 = 0.2 * LI.normal_field(71, shape, 2000)
    e, u, v = orc.apply([e0, u0, v0], "swe_flux", PRM, 60)
    assert abs(e.sum() - e0.sum()) <= 1e-13 * np.abs(e0).sum()
    # the momentum equations are not in conservation form: a change is expected
    assert abs(u.sum() - u0.sum()) > 1e-6


def _symbol(kx, ky, dt, g, f, H, U0, V0):
    """One-step Jacobian of swe_flux about (eta, u, v) = (0, U0, V0) for the
    mode exp(i (kx i + ky j)); rows/columns (eta, u, v)."""
    Sx, Sy = np.exp(1j * kx), np.exp(1j * ky)
    adv = dt * U0 * 0.5 * (Sx - 1 / Sx) + dt * V0 * 0.5 * (Sy - 1 / Sy)
    A = np.zeros((3, 3), dtype=complex)
    A[0, 0] = 1 - dt * (1 - 1 / Sx) * U0 * 0.5 * (1 + Sx) - dt * (1 - 1 / Sy) * V0 * 0.5 * (1 + Sy)
    A[0, 1] = -dt * H * (1 - 1 / Sx)
    A[0, 2] = -dt * H * (1 - 1 / Sy)
    A[1, 0] = -dt * g * (Sx - 1)
    A[1, 1] = 1 - adv
    A[1, 2] = dt * f * 0.25 * (1 + Sx) * (1 + 1 / Sy)
    A[2, 0] = -dt * g * (Sy - 1)
    A[2, 1] = -dt * f * 0.25 * (1 + 1 / Sx) * (1 + Sy)
    A[2, 2] = 1 - adv
    return A


def _apply_symbol(fields, A_of_k, power=1):
    ny, nx = fields[0].shape
    hat = np.stack([np.fft.fft2(x) for x in fields])  # (3, ny, nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    out = np.zeros_like(hat)
    for a in range(ny):
        for b in range(nx):
            A = np.linalg.matrix_power(A_of_k(kx[b], ky[a]), power)
            out[:, a, b] = A @ hat[:, a, b]
    return [np.real(np.fft.ifft2(out[k])) for k in range(3)]


@pytest.mark.parametrize("U0,V0,f", [(0.3, -0.2, 0.5), (0.0, 0.0, 1.5), (-0.4, 0.25, 0.0)])
def test_swe_flux_linearisation_matches_fourier_symbol(orc, U0, V0, f):
    dt, g, _, H = PRM
    prm = [dt, g, f, H]
    shape = (12, 10)
    m = [LI.normal_field(5, shape, k * 120) for k in range(3)]
    base = [np.zeros(shape), np.full(shape, U0), np.full(shape, V0)]
    eps = 1e-3
    plus = orc.apply([b + eps * x for b, x in zip(base, m)], "swe_flux", prm, 1)
    minus = orc.apply([b - eps * x for b, x in zip(base, m)], "swe_flux", prm, 1)
    # one step is a quadratic polynomial of the state: the central difference is exact
    jm = [(p - q) / (2 * eps) for p, q in zip(plus, minus)]
    want = _apply_symbol(m, lambda kx, ky: _symbol(kx, ky, dt, g, f, H, U0, V0))
    for k in range(3):
        assert normwise(jm[k], want[k]) <= 1e-10, k


def test_swe_flux_linearisation_many_steps(orc):
    # with f = 0 a uniform flow is steady, so T steps linearise to A(k)^T
    dt, g, _, H = PRM
    U0, V0, T = 0.25, 0.15, 20
    prm = [dt, g, 0.0, H]
    shape = (8, 12)
    m = [LI.normal_field(9, shape, k * 96) for k in range(3)]
    base = [np.zeros(shape), np.full(shape, U0), np.full(shape, V0)]
    eps = 1e-5
    plus = orc.apply([b + eps * x for b, x in zip(base, m)], "swe_flux", prm, T)
    minus = orc.apply([b - eps * x for b, x in zip(base, m)], "swe_flux", prm, T)
    jm = [(p - q) / (2 * eps) for p, q in zip(plus, minus)]
    want = _apply_symbol(m, lambda kx, ky: _symbol(kx, ky, dt, g, 0.0, H, U0, V0), power=T)
    for k in range(3):
        assert normwise(jm[k], want[k]) <= 1e-6, k


@pytest.mark.parametrize("axis", ["x", "y"])
def test_swe_flux_self_advection_closed_form(orc, axis):
    """1D wave along one axis: eta = a cos(k s), velocity along s = b cos(k s)."""
    dt, g, _, H = 0.05, 2.0, 0.0, 1.5
    prm = [dt, g, 0.0, H]
    n, p_, a, b = 16, 3, 0.3, 0.4
    k = 2 * np.pi * p_ / n
    shape = (5, n) if axis == "x" else (n, 5)
    j, i = _grid(shape)
    s = i if axis == "x" else j
    eta = a * np.cos(k * s)
    vel = b * np.cos(k * s)
    zero = np.zeros(shape)
    ins = [eta, vel, zero] if axis == "x" else [eta, zero, vel]
    e1, u1, v1 = orc.apply(ins, "swe_flux", prm, 1)
    # flux difference: H b (cos ks - cos k(s-1)) + (ab/2) cos(k/2) (cos k(2s+1/2) - cos k(2s-3/2))
    dflux = (H * b * (-2 * np.sin(k * (s - 0.5)) * np.sin(k / 2))
             + 0.5 * a * b * np.cos(k / 2) * (-2 * np.sin(k * (2 * s - 0.5)) * np.sin(k)))
    want_e = eta - dt * dflux
    # d eta to the next centre and the self-advection term vel * D vel
    d_eta = -2 * a * np.sin(k * (s + 0.5)) * np.sin(k / 2)
    adv = -0.5 * b * b * np.sin(2 * k * s) * np.sin(k)
    want_vel = vel - dt * (g * d_eta + adv)
    got_vel, got_other = (u1, v1) if axis == "x" else (v1, u1)
    assert np.max(np.abs(e1 - want_e)) <= 1e-15
    assert np.max(np.abs(got_vel - want_vel)) <= 1e-15
    assert np.max(np.abs(got_other)) == 0.0


def test_swe_flux_cross_advection_closed_form(orc):
    """u = b cos(ky j), v = c cos(kx i): only the averaged cross-advection acts."""
    dt, g, f, H = 0.05, 1.0, 0.0, 1.0
    ny, nx = 12, 10
    ky, kx = 2 * np.pi * 5 / ny, 2 * np.pi * 3 / nx
    b, c = 0.6, -0.35
    j, i = _grid((ny, nx))
    u0 = b * np.cos(ky * j)
    v0 = c * np.cos(kx * i)
    e1, u1, v1 = orc.apply([np.zeros((ny, nx)), u0, v0], "swe_flux", [dt, g, f, H], 1)
    # vbar at the u face (i+1/2, j) = c cos(kx/2) cos(kx (i+1/2)); D_y u = -b sin(ky) sin(ky j)
    want_u = u0 + dt * c * np.cos(kx / 2) * np.cos(kx * (i + 0.5)) * b * np.sin(ky) * np.sin(ky * j)
    # ubar at the v face (i, j+1/2) = b cos(ky/2) cos(ky (j+1/2)); D_x v = -c sin(kx) sin(kx i)
    want_v = v0 + dt * b * np.cos(ky / 2) * np.cos(ky * (j + 0.5)) * c * np.sin(kx) * np.sin(kx * i)
    assert np.max(np.abs(e1)) <= 1e-15
    assert np.max(np.abs(u1 - want_u)) <= 1e-15
    assert np.max(np.abs(v1 - want_v)) <= 1e-15


def test_swe_flux_coriolis_corner_closed_form(orc):
    """v = c cos(kx i + ky j) alone, f != 0: u' = dt f vbar, vbar from the four
    v faces (i,j), (i+1,j), (i,j-1), (i+1,j-1) around the u face."""
    dt, g, f, H = 0.05, 1.0, 0.8, 1.0
    ny, nx = 9, 14
    kx, ky = 2 * np.pi * 4 / nx, 2 * np.pi * 2 / ny
    c = 0.5
    j, i = _grid((ny, nx))
    v0 = c * np.cos(kx * i + ky * j)
    e1, u1, v1 = orc.apply([np.zeros((ny, nx)), np.zeros((ny, nx)), v0], "swe_flux",
                           [dt, g, f, H], 1)
    # (1 + Sx)(1 + 1/Sy)/4 acting on exp(i theta): cos(kx/2) cos(ky/2) exp(i(theta + kx/2 - ky/2))
    vbar = c * np.cos(kx / 2) * np.cos(ky / 2) * np.cos(kx * i + ky * j + kx / 2 - ky / 2)
    assert np.max(np.abs(u1 - dt * f * vbar)) <= 1e-15
    # v' = v - dt v D_y v (self-advection in y) and eta' from the flux of v
    dyv = -c * np.sin(ky) * np.sin(kx * i + ky * j)
    assert np.max(np.abs(v1 - (v0 - dt * v0 * dyv))) <= 1e-15


# ---------------------------------------------------------------- Runge-Kutta
def _rk_poly(z, stages):
    return 1 + z + z * z / 2 + (z ** 3 / 6 if stages == 3 else 0)


@pytest.mark.parametrize("scheme,stages", [("rk2", 2), ("rk3", 3)])
def test_rk_fourier_mode_stability_polynomial(orc, scheme, stages):
    n, c, T = 32, 0.2, 30
    j, i = _grid((n, n))
    for p, q in ((1, 0), (3, 5), (16, 16)):
        mode = np.cos(2 * np.pi * (p * i + q * j) / n)
        z = -4 * c * (np.sin(np.pi * p / n) ** 2 + np.sin(np.pi * q / n) ** 2)
        got = orc.apply(mode, "jacobi5", [c], T, scheme=scheme)
        assert np.max(np.abs(got - _rk_poly(z, stages) ** T * mode)) <= 1e-13


def test_rk3_dirichlet_sine_mode(orc):
    n, c, T = 10, 0.1, 12
    idx = np.arange(1, n + 1)
    pz, py, px = 1, 2, 3
    mode = (np.sin(np.pi * pz * idx / (n + 1))[:, None, None]
            * np.sin(np.pi * py * idx / (n + 1))[None, :, None]
            * np.sin(np.pi * px * idx / (n + 1))[None, None, :])
    z = -4 * c * sum(np.sin(np.pi * p / (2 * (n + 1))) ** 2 for p in (pz, py, px))
    got = orc.apply(mode, "diff7", [c], T, bc=[1, 1, 1], scheme="rk3")
    assert np.max(np.abs(got - _rk_poly(z, 3) ** T * mode)) <= 1e-14


@pytest.mark.parametrize("scheme,stages", [("rk2", 2), ("rk3", 3)])
def test_rk_swe_flux_uniform_state(orc, scheme, stages):
    dt, g, f, H = PRM
    shape, T = (5, 6), 40
    U0, V0 = -0.3, 0.9
    e, u, v = orc.apply([np.full(shape, 0.2), np.full(shape, U0), np.full(shape, V0)],
                        "swe_flux", PRM, T, scheme=scheme)
    Z = dt * f * np.array([[0.0, 1.0], [-1.0, 0.0]])
    P = np.eye(2) + Z + Z @ Z / 2 + (Z @ Z @ Z / 6 if stages == 3 else 0)
    want = np.linalg.matrix_power(P, T) @ np.array([U0, V0])
    assert np.max(np.abs(e - 0.2)) <= 1e-15
    assert np.max(np.abs(u - want[0])) <= 1e-14 and np.max(np.abs(v - want[1])) <= 1e-14


def test_rk3_swe_flux_conserves_mass(orc):
    shape = (16, 18)
    fields = [0.1 * LI.normal_field(3, shape), 0.2 * LI.normal_field(3, shape, 500),
              0.2 * LI.normal_field(3, shape, 1000)]
    e, _, _ = orc.apply(fields, "swe_flux", PRM, 30, scheme="rk3")
    assert abs(e.sum() - fields[0].sum()) <= 1e-13 * np.abs(fields[0]).sum()


@pytest.mark.parametrize("scheme,stages", [("rk2", 2), ("rk3", 3)])
def test_rk_box_stencil_bruteforce(orc, scheme, stages):
    """Dense Euler matrix M of an asymmetric box table on a mixed-BC grid; the
    scheme's step is I + Z + Z^2/2 (+ Z^3/6) with Z = M - I."""
    rng = np.random.default_rng(4)
    w = rng.normal(size=(3, 3)) * 0.15
    shape = (6, 7)
    bc = [(0, 0), (1, 1)]  # y periodic, x Dirichlet 0
    M, b = assemble(shape, taps("linear", weights_table=w), bc=bc, bval=[0.0, 0.0])
    assert np.all(b == 0)
    Z = M - np.eye(M.shape[0])
    P = np.eye(M.shape[0]) + Z + Z @ Z / 2 + (Z @ Z @ Z / 6 if stages == 3 else 0)
    u0 = LI.uniform_field(8, shape)
    T = 7
    want = (np.linalg.matrix_power(P, T) @ u0.ravel()).reshape(shape)
    got = orc.apply(u0, "linear", nsteps=T, bc=bc, weights_table=w, scheme=scheme)
    assert normwise(got, want) <= 1e-13


def test_rk_euler_scheme_is_plain_apply(orc):
    u0 = LI.uniform_field(2, (9, 11))
    a = orc.apply(u0, "jacobi5", [0.2], 5)
    b = orc.apply(u0, "jacobi5", [0.2], 5, scheme="euler")
    assert np.array_equal(a, b)
