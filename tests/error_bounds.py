"""Error bounds of FP32 / BF16 storage runs against the FP64 oracle, derived
from the arithmetic of each local function (test infrastructure).

A run stores x_{t+1} = fl(F(x_t)); the oracle computes y_{t+1} = F(y_t) in
FP64 from the same stored input.  With e_t = x_{t+1} - F(x_t) the local error
of one step, the global error obeys E_{t+1} = F(x_t) - F(y_t) + e_t.

* Local error.  Each function below follows the operation tree of one step of
  a builtin (the functors in the library evaluate exactly these operations,
  each rounded once, FMAs once): with u the unit roundoff of FP32 (2^-24), an
  operation whose exact result is r commits at most u |r|, and a coefficient
  stored in FP32 differs from its FP64 value by at most u times its size.
  Summing the first-order contributions, with every intermediate bounded
  through the field magnitudes M_f, gives eps_f >= |e_t| for field f.  BF16
  storage adds the final rounding to bfloat16, at most half an ulp of the
  largest stored value (unit roundoff 2^-8).
* Propagation, linear functions.  E_T = sum_s A^s e_{T-1-s}, so
  |E_T,i|_inf <= sum_s sum_j ||K^s_{j->i}||_1 eps_j, where K^s_{j->i} is the
  response of field i to a unit impulse in field j after s exact steps (the
  oracle applied to impulses on a periodic grid wide enough that nothing
  wraps).  On a Dirichlet grid the same weights act with some taps dropped;
  for the non-negative-weight functions used there the impulse norms are 1
  either way.
* Mean of a conservative field.  Where the exact step conserves the mean of a
  field (periodic shallow water: every field), |mean(E_T,i)| <= T eps_i,
  without amplification: a systematic bias of about an ulp per step exceeds it.
* Propagation, non-linear functions.  |E_{t+1}| <= |J_t| |E_t| + eps_t
  elementwise to first order, with J_t the step's Jacobian on the oracle's
  state y_t; the bound B_t is propagated with |J_t| alongside the oracle run
  (a 1 % margin covers the second-order terms at these error sizes).
"""
from __future__ import annotations

import math

import numpy as np

U32 = 2.0 ** -24   # FP32 unit roundoff
U_BF16 = 2.0 ** -8  # bfloat16 unit roundoff (8 significant bits)


def half_ulp(m: float, dtype: str) -> float:
    """Half an ulp of a value of magnitude m (the largest rounding error of
    storing any value of magnitude <= m)."""
    if m <= 0:
        return 0.0
    p = {"f32": 24, "bf16": 8, "f64": 53}[dtype]
    e = math.floor(math.log2(m))
    return 2.0 ** (e - p)


# ------------------------------------------------------------------ local errors
def local_eps(kind: str, prm, M, dtype: str, dh: float | None = None):
    """Per-field bound of one step's local error for builtin `kind`.  M: per
    field, a bound of |value| over the states of the run (inputs and outputs
    of every step).  dh (swe_cgrid): a bound of the differences |h(i+1,j) -
    h(i,j)| and |h(i,j+1) - h(i,j)| over the run (default 2 M_h)."""
    u = U32
    if kind == "diff7":
        # nb = ((W+E)+(S+N))+(D+U): partial sums <= 2,2,4,2,6 M -> 16 M u;
        # L = fma(-6, x, nb), |L| <= 12 M -> 12 M u; o = fma(c32, L, x): c32
        # error u c 12 M, c (16 + 12) M u, final u |o| <= u ||A||_inf M.
        c = prm[0]
        m = M[0]
        eps = [u * m * (abs(c) * 12 + abs(c) * 28 + abs(1 - 6 * c) + 6 * abs(c))]
    elif kind == "jacobi5":
        # nb = (W+E)+(S+N): 2,2,4 M -> 8 M u; L = fma(-4, x, nb), |L| <= 8 M;
        # o = fma(c32, L, x)
        c = prm[0]
        m = M[0]
        eps = [u * m * (abs(c) * 8 + abs(c) * 16 + abs(1 - 4 * c) + 4 * abs(c))]
    elif kind == "star9r2":
        # s1, s2: 8 M u each (|s| <= 4 M); m5 = -5 x: 5 M u; a = fma(k2, s2, m5),
        # |a| <= 16/3 M; lap = fma(k1, s1, a), |lap| <= 32/3 M; o = fma(c32,
        # lap, x), |o| <= ||A||_inf M.
        c = prm[0]
        m = M[0]
        err_a = m * (4.0 / 12 + 8.0 / 12 + 5 + 16.0 / 3)
        err_lap = m * (4.0 / 3 * 4 + 4.0 / 3 * 8) + err_a + m * 32.0 / 3
        norm_a = abs(1 - 5 * c) + abs(c) * (16.0 / 3 + 1.0 / 3)
        eps = [u * (abs(c) * m * 32.0 / 3 + abs(c) * err_lap + m * norm_a)]
    elif kind == "swe_cgrid":
        # h' = fma(c1, (u - uW) + (v - vS), h): differences <= 2 Muv each, sum
        # <= 4 Muv, 8 Muv u in all; c1 = fl(-dt H).  u' = fma(c2, hE - h, u):
        # coefficient u dt g dh, difference rounded once (u dh), final u Muv.
        dt, g, H = prm
        mh, muv = M[0], max(M[1], M[2])
        d = 2 * mh if dh is None else dh
        e_h = u * (dt * H * 4 * muv + dt * H * 8 * muv + mh)
        e_u = u * (dt * g * d + dt * g * d + muv)
        eps = [e_h, e_u, e_u]
    else:
        raise ValueError(kind)
    if dtype == "bf16":
        eps = [e + half_ulp(m, "bf16") for e, m in zip(eps, M)]
    elif dtype != "f32":
        raise ValueError(dtype)
    return np.array(eps)


def local_eps_gray_scott(prm, mu: float, mv: float, dtype: str = "f32"):
    """Local error of one Gray-Scott step (the GRAY_SCOTT body in
    user_bodies.py; P = dt, Du, Dv, F, k, all held in FP32) for |u| <= mu,
    |v| <= mv:
      lu = fma(-4, u, (uW+uE)+(uS+uN))            |lu| <= 8 mu
      vv = v*v, uvv = u*vv                          |uvv| <= mu mv^2
      r_u = fma(F, 1 - u, -uvv)                     |r_u| <= F (1 + mu) + mu mv^2
      t_u = fma(Du, lu, r_u);  u' = fma(dt, t_u, u)
      r_v = fma(-(F + k), v, uvv)                   |r_v| <= (F + k) mv + mu mv^2
      t_v = fma(Dv, lv, r_v);  v' = fma(dt, t_v, v)."""
    dt, Du, Dv, F, k = prm
    u = U32
    uvv = mu * mv * mv
    e_uvv = u * 2 * uvv
    e_lu, e_lv = u * 16 * mu, u * 16 * mv
    r_u = F * (1 + mu) + uvv
    e_ru = u * F * (1 + mu) + F * u * (1 + mu) + e_uvv + u * r_u
    t_u = Du * 8 * mu + r_u
    e_tu = u * Du * 8 * mu + Du * e_lu + e_ru + u * t_u
    Fk = F + k
    r_v = Fk * mv + uvv
    e_rv = u * 2 * Fk * mv + e_uvv + u * r_v
    t_v = Dv * 8 * mv + r_v
    e_tv = u * Dv * 8 * mv + Dv * e_lv + e_rv + u * t_v
    eps_u = u * dt * t_u + dt * e_tu + u * (mu + dt * t_u)
    eps_v = u * dt * t_v + dt * e_tv + u * (mv + dt * t_v)
    if dtype == "bf16":
        eps_u += half_ulp(mu, "bf16")
        eps_v += half_ulp(mv, "bf16")
    return eps_u, eps_v


# ------------------------------------------------------------------ propagation
def impulse_norms(orc, kind: str, prm, nf: int, ndim: int, radius: int, T: int):
    """norms[s, i, j] = ||K^s_{j->i}||_1 for s = 0..T-1 (exact FP64 steps by the
    oracle on a periodic grid of side 2 R T + 3 around a unit impulse)."""
    n = 2 * radius * T + 3
    shape = (n,) * ndim
    centre = (n // 2,) * ndim
    resp = []
    for j in range(nf):
        f = [np.zeros(shape) for _ in range(nf)]
        f[j][centre] = 1.0
        resp.append(f)
    out = np.zeros((T, nf, nf))
    nth = orc.max_threads()
    for s in range(T):
        for j in range(nf):
            for i in range(nf):
                out[s, i, j] = np.abs(resp[j][i]).sum()
        if s + 1 < T:
            nxt = []
            for r in resp:
                y = orc.apply(r if nf > 1 else r[0], kind, prm, 1, nthreads=nth)
                nxt.append(y if nf > 1 else [y])
            resp = nxt
    return out


def sup_bound(norms: np.ndarray, eps) -> np.ndarray:
    """Per field: sum_s sum_j norms[s, i, j] eps_j."""
    return np.einsum("sij,j->i", norms, np.asarray(eps, dtype=np.float64))


def growth(norms: np.ndarray) -> float:
    """Largest ||A^s||_inf over the run (bounds every intermediate state)."""
    return float(norms.sum(axis=2).max())


def gray_scott_majorant(orc, body: str, prm, fields0, T: int, dtype: str = "f32",
                        bc=None, bval=None):
    """Elementwise first-order bound B_T >= |x_T - y_T| for the Gray-Scott
    body, propagated with |J_t| along the oracle's trajectory from the stored
    input `fields0` (two FP64 arrays); returns (B_u, B_v) and y_T.  Periodic
    grids only (|J| taps wrap)."""
    dt, Du, Dv, F, k = prm
    y = [np.asarray(f, dtype=np.float64).copy() for f in fields0]
    B = [np.zeros_like(y[0]), np.zeros_like(y[1])]
    nth = orc.max_threads()

    def nbsum(a):
        return (np.roll(a, 1, 0) + np.roll(a, -1, 0) + np.roll(a, 1, 1) + np.roll(a, -1, 1))

    for _ in range(T):
        yn = orc.apply_source(y, body, prm, 1, bc=bc, bval=bval, nthreads=nth)
        # magnitudes over this step's input and output (the stored run stays
        # within B of the oracle's)
        mu = max(np.max(np.abs(y[0]) + B[0]), np.max(np.abs(yn[0])) + np.max(B[0]))
        mv = max(np.max(np.abs(y[1]) + B[1]), np.max(np.abs(yn[1])) + np.max(B[1]))
        eu, ev = local_eps_gray_scott(prm, mu, mv, dtype)
        uu, vv = y
        # |J_t| applied to B: the centre and neighbour weights of each row
        cu = np.abs(1 - 4 * dt * Du - dt * (F + vv * vv))
        cv = np.abs(1 - 4 * dt * Dv + dt * (2 * uu * vv - (F + k)))
        Bu = cu * B[0] + dt * Du * nbsum(B[0]) + np.abs(2 * dt * uu * vv) * B[1] + eu
        Bv = cv * B[1] + dt * Dv * nbsum(B[1]) + dt * vv * vv * B[0] + ev
        B = [Bu * 1.01, Bv * 1.01]
        y = [np.asarray(a, dtype=np.float64) for a in yn]
    return B, y
