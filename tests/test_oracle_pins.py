"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks the oracle against a value printed in the paper (golden
fixtures), a closed form (Fourier / sine eigenmodes, FFT and DST whole-field
solutions), a brute-force dense operator assembled independently
(tests/dense_ref.py), or an exact invariant.  The cases are chosen so that a
dropped term, a wrong sign or index, or a transposed operand fails at least
one of them.
"""
import os

import numpy as np
import pytest
import scipy.fft as sfft

import lope_inputs as LI
from dense_ref import assemble, laplacian_taps, normwise, read_blocks, swe_matrix, taps

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generators
def test_splitmix64_known_outputs():
    with open(os.path.join(GOLD, "splitmix64.txt")) as fh:
        want = [int(l, 16) for l in fh if l.strip() and not l.startswith("#")]
    got = [int(x) for x in LI.splitmix64(0, 3)]
    assert got == want


def test_uniform_and_normal_moments():
    u = LI.uniform(7, 400_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3
    z = LI.normal(7, 400_000)
    assert abs(z.mean()) < 5e-3 and abs(z.std() - 1.0) < 5e-3


def test_bf16_rounding_ties_to_even():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -30, -2.5])
    got = LI.round_to_bf16(x)
    assert list(got) == [1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5]


# ---------------------------------------------------------------- paper values
def test_fig1_impulse_golden(orc):
    inp, out = read_blocks(os.path.join(GOLD, "fig1_impulse.txt"))
    got = orc.apply(inp, "jacobi5", [1.0], 1)
    assert np.array_equal(got, out)


def test_index_orientation_golden(orc):
    inp, right, above = read_blocks(os.path.join(GOLD, "index_orientation.txt"))
    w = np.zeros((3, 3))
    w[1, 2] = 1.0  # (dy=0, dx=+1): U(+1,0)
    assert np.array_equal(orc.apply(inp, "linear", nsteps=1, weights_table=w), right)
    w = np.zeros((3, 3))
    w[2, 1] = 1.0  # (dy=+1, dx=0): U(0,+1)
    assert np.array_equal(orc.apply(inp, "linear", nsteps=1, weights_table=w), above)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("p,q", [(1, 0), (3, 5), (128, 128), (7, 200)])
def test_jacobi5_fourier_mode_256(orc, p, q):
    """A periodic Fourier mode is scaled by g = 1 - 4c(sin^2(pi p/N) + sin^2(pi q/N)) per step."""
    n, c, T = 256, 0.2, 100
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u0 = np.cos(2 * np.pi * (p * i / n + q * j / n))
    g = 1.0 - 4.0 * c * (np.sin(np.pi * p / n) ** 2 + np.sin(np.pi * q / n) ** 2)
    got = orc.apply(u0, "jacobi5", [c], T)
    assert np.max(np.abs(got - g ** T * u0)) <= 1e-12 * max(abs(g) ** T, 1e-300) + 1e-13


def test_jacobi5_fft_whole_field(orc):
    """Random field on a non-square periodic grid against FFT2 * g(k)^T."""
    ny, nx, c, T = 48, 64, 0.2, 37
    u0 = LI.uniform_field(11, (ny, nx))
    ky = 2 * np.pi * np.fft.fftfreq(ny)[:, None]
    kx = 2 * np.pi * np.fft.fftfreq(nx)[None, :]
    g = 1.0 - 4.0 * c * (np.sin(ky / 2) ** 2 + np.sin(kx / 2) ** 2)
    want = np.real(np.fft.ifft2(np.fft.fft2(u0) * g ** T))
    got = orc.apply(u0, "jacobi5", [c], T)
    assert normwise(got, want) < 1e-12


def test_star9r2_fft_whole_field(orc):
    """lambda(k) = -5/2 + (8/3)cos k - (1/6)cos 2k per axis."""
    ny, nx, c, T = 40, 32, 0.1, 25
    u0 = LI.uniform_field(12, (ny, nx))
    lam = lambda k: -2.5 + (8.0 / 3.0) * np.cos(k) - (1.0 / 6.0) * np.cos(2 * k)
    ky = 2 * np.pi * np.fft.fftfreq(ny)[:, None]
    kx = 2 * np.pi * np.fft.fftfreq(nx)[None, :]
    g = 1.0 + c * (lam(ky) + lam(kx))
    want = np.real(np.fft.ifft2(np.fft.fft2(u0) * g ** T))
    got = orc.apply(u0, "star9r2", [c], T)
    assert normwise(got, want) < 1e-12


def test_diff7_dirichlet_sine_mode(orc):
    """Sine modes are eigenvectors of the Dirichlet-0 operator."""
    shape = (9, 10, 12)
    p = (2, 3, 5)
    c, T = 0.1, 30
    grids = np.meshgrid(*[np.arange(1, s + 1) for s in shape], indexing="ij")
    u0 = np.ones(shape)
    g = 1.0
    for ax in range(3):
        u0 = u0 * np.sin(np.pi * p[ax] * grids[ax] / (shape[ax] + 1))
        g -= 4 * c * np.sin(np.pi * p[ax] / (2 * (shape[ax] + 1))) ** 2
    got = orc.apply(u0, "diff7", [c], T, bc=[1, 1, 1])
    assert np.max(np.abs(got - g ** T * u0)) < 1e-13


def test_diff7_dirichlet_dst_whole_field(orc):
    """Random field against an orthonormal DST-I solution (Dirichlet 0)."""
    shape = (7, 11, 13)
    c, T = 0.1, 20
    u0 = LI.uniform_field(13, shape)
    coef = sfft.dstn(u0, type=1, norm="ortho")
    g = np.ones(shape)
    for ax, s in enumerate(shape):
        k = np.arange(1, s + 1) * np.pi / (s + 1)
        sh = [1, 1, 1]
        sh[ax] = s
        g = g - 4 * c * np.sin(k / 2).reshape(sh) ** 2
    want = sfft.idstn(coef * g ** T, type=1, norm="ortho")
    got = orc.apply(u0, "diff7", [c], T, bc=[1, 1, 1])
    assert normwise(got, want) < 1e-12


def test_swe_fft_whole_field(orc):
    """Per wavenumber, the C-grid update is a 3x3 matrix G(k) = I + dt A(k)."""
    ny, nx, T = 16, 24, 50
    dt, gr, H = 0.02, 1.0, 1.0
    h, u, v = LI.swe_fields(14, (ny, nx))
    ky = 2 * np.pi * np.fft.fftfreq(ny)[:, None] * np.ones((1, nx))
    kx = 2 * np.pi * np.fft.fftfreq(nx)[None, :] * np.ones((ny, 1))
    ex, ey = np.exp(1j * kx), np.exp(1j * ky)
    G = np.zeros((ny, nx, 3, 3), dtype=complex)
    G[..., 0, 0] = G[..., 1, 1] = G[..., 2, 2] = 1.0
    G[..., 0, 1] = -dt * H * (1 - 1 / ex)
    G[..., 0, 2] = -dt * H * (1 - 1 / ey)
    G[..., 1, 0] = -dt * gr * (ex - 1)
    G[..., 2, 0] = -dt * gr * (ey - 1)
    GT = np.linalg.matrix_power(G, T)
    s = np.stack([np.fft.fft2(f) for f in (h, u, v)], axis=-1)
    sT = np.einsum("...ij,...j->...i", GT, s)
    want = [np.real(np.fft.ifft2(sT[..., k])) for k in range(3)]
    got = orc.apply([h, u, v], "swe_cgrid", [dt, gr, H], T)
    for k in range(3):
        assert normwise(got[k], want[k]) < 1e-12


# ---------------------------------------------------------------- brute force
def _dense_power(M, b, u0, T):
    u = u0.ravel().copy()
    for _ in range(T):
        u = M @ u + b
    return u.reshape(u0.shape)


@pytest.mark.parametrize(
    "kind,shape,c,bc,bval",
    [
        ("jacobi5", (8, 8), 0.2, [0, 0], None),
        ("jacobi5", (8, 8), 0.2, [1, 1], [0.7, -0.3]),
        ("jacobi5", (8, 6), 0.2, [0, (1, 1)], [0.0, (0.5, -1.5)]),
        ("diff7", (4, 4, 4), 0.1, [0, 0, 0], None),
        ("diff7", (4, 5, 3), 0.1, [1, 0, 1], [2.0, 0.0, -1.0]),
        ("star9r2", (8, 8), 0.1, [0, 0], None),
        ("star9r2", (8, 7), 0.1, [1, 1], [0.25, 0.25]),
    ],
)
def test_bruteforce_forward(orc, kind, shape, c, bc, bval):
    M, b = assemble(shape, taps(kind, c), bc, bval)
    u0 = LI.uniform_field(21, shape)
    got = orc.apply(u0, kind, [c], 9, bc=bc, bval=bval)
    assert normwise(got, _dense_power(M, b, u0, 9)) < 1e-14


@pytest.mark.parametrize("ndim,r,bc", [(2, 1, [1, 0]), (2, 2, [0, 0]), (3, 1, [0, 1, 0])])
def test_bruteforce_linear_asymmetric(orc, ndim, r, bc):
    """A random asymmetric box stencil with corners pins offset orientation."""
    side = 2 * r + 1
    w = LI.uniform_field(31 + ndim + r, (side,) * ndim) - 0.5
    shape = (6, 7) if ndim == 2 else (5, 4, 6)
    bval = [0.3] * ndim
    M, b = assemble(shape, taps("linear", weights_table=w, ndim=ndim), bc, bval)
    u0 = LI.uniform_field(22, shape)
    got = orc.apply(u0, "linear", nsteps=3, bc=bc, bval=bval, weights_table=w)
    assert normwise(got, _dense_power(M, b, u0, 3)) < 1e-13


def test_bruteforce_swe(orc):
    shape = (8, 8)
    dt, gr, H = 0.02, 1.0, 1.0
    M = swe_matrix(shape, dt, gr, H)
    h, u, v = LI.swe_fields(23, shape)
    x = np.concatenate([h.ravel(), u.ravel(), v.ravel()])
    for _ in range(11):
        x = M @ x
    got = orc.apply([h, u, v], "swe_cgrid", [dt, gr, H], 11)
    n = h.size
    for k in range(3):
        assert normwise(got[k].ravel(), x[k * n:(k + 1) * n]) < 1e-14


@pytest.mark.parametrize(
    "kind,shape,c,bc,bval",
    [
        ("jacobi5", (8, 8), 0.2, [0, 0], None),
        ("jacobi5", (6, 8), 0.2, [1, 1], [0.4, 0.4]),
        ("diff7", (4, 4, 4), 0.1, [0, 0, 0], None),
        ("diff7", (4, 3, 5), 0.1, [1, 1, 0], [0.0, 0.0, 0.0]),
        ("star9r2", (8, 8), 0.1, [0, 0], None),
    ],
)
def test_bruteforce_adjoint(orc, kind, shape, c, bc, bval):
    """dL/du0 = (M^T)^T lamT and dL/dc = sum_t <lam_{t+1}, L u_t + b_L>."""
    T = 6
    M, b = assemble(shape, taps(kind, c), bc, bval)
    Lm, bL = assemble(shape, laplacian_taps(kind), bc, bval)
    u0 = LI.uniform_field(24, shape)
    lamT = LI.normal_field(25, shape)
    traj = [u0.ravel()]
    for _ in range(T):
        traj.append(M @ traj[-1] + b)
    lam = lamT.ravel().copy()
    gc = 0.0
    for t in range(T - 1, -1, -1):
        gc += lam @ (Lm @ traj[t] + bL)
        lam = M.T @ lam
    g, gc_or = orc.vjp(u0, lamT, kind, [c], T, bc=bc, bval=bval)
    assert normwise(g.ravel(), lam) < 1e-13
    assert abs(gc_or - gc) <= 1e-12 * abs(gc)


def test_weights_table_matches_dense(orc):
    """The oracle's weight table reproduces the dense operator's rows."""
    for kind, ndim, c in (("jacobi5", 2, 0.2), ("diff7", 3, 0.1), ("star9r2", 2, 0.1)):
        w = orc.weights(kind, [c], ndim)
        shape = (9,) * ndim
        M1, _ = assemble(shape, taps(kind, c), None, None)
        M2, _ = assemble(shape, taps("linear", weights_table=w, ndim=ndim), None, None)
        assert np.array_equal(M1, M2)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("kind,shape,prm", [("jacobi5", (10, 12), [0.2]),
                                             ("diff7", (5, 6, 7), [0.1]),
                                             ("star9r2", (9, 11), [0.1])])
def test_constant_field_and_sum(orc, kind, shape, prm):
    const = np.full(shape, 0.375)
    assert np.array_equal(orc.apply(const, kind, prm, 5), const)
    u0 = LI.uniform_field(41, shape)
    u = orc.apply(u0, kind, prm, 15)
    assert abs(u.sum() - u0.sum()) < 1e-11 * u0.size


def test_swe_conservation(orc):
    h, u, v = LI.swe_fields(42, (20, 18))
    out = orc.apply([h, u, v], "swe_cgrid", [0.02, 1.0, 1.0], 40)
    for a, b in zip((h, u, v), out):
        assert abs(a.sum() - b.sum()) < 1e-11 * a.size


def test_linearity(orc):
    shape = (6, 7, 8)
    x = LI.uniform_field(43, shape)
    y = LI.normal_field(44, shape)
    a, b = 0.7, -1.3
    lhs = orc.apply(a * x + b * y, "diff7", [0.1], 4, bc=[1, 0, 1])
    rhs = a * orc.apply(x, "diff7", [0.1], 4, bc=[1, 0, 1]) + b * orc.apply(y, "diff7", [0.1], 4, bc=[1, 0, 1])
    assert normwise(lhs, rhs) < 1e-14


def test_dot_product_identity(orc):
    """<A x, y> = <x, A^T y> between the forward gather and the scatter adjoint."""
    for kind, shape, c, bc in (("diff7", (6, 5, 7), 0.1, [0, 1, 0]), ("star9r2", (10, 9), 0.1, [0, 0]),
                               ("jacobi5", (7, 9), 0.2, [1, 1])):
        x = LI.uniform_field(45, shape)
        y = LI.normal_field(46, shape)
        Ax = orc.apply(x, kind, [c], 3, bc=bc)
        ATy, _ = orc.vjp(x, y, kind, [c], 3, bc=bc)
        assert abs(np.vdot(Ax, y) - np.vdot(x, ATy)) < 1e-13 * x.size


def test_adjoint_single_mode_closed_form(orc):
    """u0 = a*m, target 0, periodic: L = a^2 g^(2T)|m|^2, dL/dc = 2 a^2 T g^(2T-1) lam_k |m|^2."""
    n, c, T, amp = 16, 0.1, 12, 0.8
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    k = 2 * np.pi / n
    m = np.cos(k * x + 2 * k * y)
    lam_k = -4 * (np.sin(k / 2) ** 2 + np.sin(k) ** 2)
    g = 1 + c * lam_k
    loss, gu, gc = orc.adjoint(amp * m, np.zeros_like(m), "diff7", [c], T)
    mm = np.vdot(m, m)
    assert abs(loss - amp ** 2 * g ** (2 * T) * mm) < 1e-12 * loss
    assert abs(gc - 2 * amp ** 2 * T * g ** (2 * T - 1) * lam_k * mm) < 1e-10 * abs(gc)
    assert np.max(np.abs(gu - 2 * g ** (2 * T) * amp * m)) < 1e-13


def test_adjoint_central_differences_32cube(orc):
    """Central differences with eps = 1e-3 in FP64 on 32^3, 100 steps.

    The loss is quadratic in u0, so the u0-directional difference is exact up to
    rounding; in c it is a polynomial and the O(eps^2) error is bounded.
    """
    n, c, T, eps = 32, 0.1, 100, 1e-3
    u0 = LI.uniform_field(1004, (n, n, n))
    tgt = LI.normal_field(2004, (n, n, n))
    d = LI.normal_field(47, (n, n, n))
    loss, gu, gc = orc.adjoint(u0, tgt, "diff7", [c], T, nthreads=4)

    def L(u, cc):
        uT = orc.apply(u, "diff7", [cc], T, nthreads=4)
        return float(np.sum((uT - tgt) ** 2))

    fd_u = (L(u0 + eps * d, c) - L(u0 - eps * d, c)) / (2 * eps)
    assert abs(fd_u - np.vdot(gu, d)) < 1e-8 * abs(fd_u)
    fd_c = (L(u0, c + eps) - L(u0, c - eps)) / (2 * eps)
    fd_c2 = (L(u0, c + eps / 2) - L(u0, c - eps / 2)) / eps
    assert abs(fd_c - gc) < 1e-3 * abs(gc)
    # Richardson extrapolation removes the O(eps^2) term of the central difference.
    assert abs((4 * fd_c2 - fd_c) / 3 - gc) < 1e-6 * abs(gc)
    assert abs(loss - L(u0, c)) < 1e-12 * loss


def test_corner_ghost_takes_the_slowest_crossed_axis(orc):
    """A corner ghost cell that crosses Dirichlet sides of several axes takes the
    value of the slowest one (z, then y, then x); a crossed periodic axis does
    not change that.  Pinned with box weights that read only one corner."""
    u = np.zeros((4, 5, 6))
    w = np.zeros((3, 3, 3))
    w[0, 0, 0] = 1.0  # the tap (dz, dy, dx) = (-1, -1, -1)
    bval = [(7.0, 0.0), (5.0, 0.0), (3.0, 0.0)]
    got = orc.apply(u, "linear", nsteps=1, bc=[1, 1, 1], bval=bval, weights_table=w)
    assert got[0, 0, 0] == 7.0  # z, y and x crossed: z decides
    assert got[1, 0, 0] == 5.0  # y and x crossed: y decides
    assert got[1, 1, 0] == 3.0  # x only
    assert got[1, 1, 1] == 0.0  # inside
    # z periodic: the wrapped z does not hide the y side's value
    got = orc.apply(u, "linear", nsteps=1, bc=[0, 1, 1], bval=[0.0, (5.0, 0.0), (3.0, 0.0)],
                    weights_table=w)
    assert got[0, 0, 0] == 5.0 and got[0, 1, 0] == 3.0
