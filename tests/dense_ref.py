"""Brute-force dense operators for tiny grids (test helper, FP64).

One step of a linear local function is u' = M u + b, where M holds the
stencil weights placed with modular (periodic) or dropped-to-constant
(Dirichlet) index arithmetic and b collects the Dirichlet halo values.  The
matrices are assembled here from each stencil's mathematical definition,
independently of the oracle's loops, so that the two can check each other.

Grids are tuples of extents, slowest axis first; offsets are given as
(dx, dy[, dz]) in the paper's local index order (first offset along the
fastest axis).
"""
from __future__ import annotations

import itertools

import numpy as np


def taps(kind, c=None, weights_table=None, ndim=2):
    """Tap list [(offset (dx,dy[,dz]), weight)] of a single-field stencil."""
    if kind == "jacobi5":
        t = [((0, 0), 1.0 - 4.0 * c)]
        t += [((dx, dy), c) for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1))]
        return t
    if kind == "diff7":
        t = [((0, 0, 0), 1.0 - 6.0 * c)]
        for ax in range(3):
            for s in (-1, 1):
                o = [0, 0, 0]
                o[ax] = s
                t.append((tuple(o), c))
        return t
    if kind == "star9r2":
        coef = {1: 4.0 / 3.0, 2: -1.0 / 12.0}
        t = [((0, 0), 1.0 - 5.0 * c)]
        for d, w in coef.items():
            for s in (-d, d):
                t.append(((s, 0), c * w))
                t.append(((0, s), c * w))
        return t
    if kind == "linear":
        w = np.asarray(weights_table, dtype=np.float64)
        r = (w.shape[0] - 1) // 2
        t = []
        for idx in itertools.product(range(2 * r + 1), repeat=ndim):
            wt = w[idx]
            if wt != 0.0:
                # idx is (dz, dy, dx) slowest first, shifted by r
                off = tuple(i - r for i in reversed(idx))
                t.append((off, float(wt)))
        return t
    raise ValueError(kind)


def laplacian_taps(kind):
    """Taps of L in u' = u + c L u, for the diffusion-form stencils."""
    if kind == "jacobi5":
        return [((0, 0), -4.0)] + [((dx, dy), 1.0) for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1))]
    if kind == "diff7":
        t = [((0, 0, 0), -6.0)]
        for ax in range(3):
            for s in (-1, 1):
                o = [0, 0, 0]
                o[ax] = s
                t.append((tuple(o), 1.0))
        return t
    if kind == "star9r2":
        t = [((0, 0), -5.0)]
        for d, w in ((1, 4.0 / 3.0), (2, -1.0 / 12.0)):
            for s in (-d, d):
                t += [((s, 0), w), ((0, s), w)]
        return t
    raise ValueError(kind)


def _bc_pairs(ndim, bc, bval):
    bc = bc if bc is not None else [0] * ndim
    bval = bval if bval is not None else [0.0] * ndim
    out = []
    for ax in range(ndim):
        k, v = bc[ax], bval[ax]
        kl, kh = (k, k) if np.isscalar(k) else k
        vl, vh = (v, v) if np.isscalar(v) else v
        out.append(((kl, kh), (vl, vh)))
    return out


def assemble(shape, tap_list, bc=None, bval=None):
    """Dense (M, b) for one step of a single-field linear stencil."""
    ndim = len(shape)
    n = int(np.prod(shape))
    M = np.zeros((n, n))
    b = np.zeros(n)
    pairs = _bc_pairs(ndim, bc, bval)
    for p in itertools.product(*[range(s) for s in shape]):
        row = np.ravel_multi_index(p, shape)
        for off, w in tap_list:
            q = list(p)
            const = None
            # offsets are (dx, dy[, dz]); axis ax (slowest first) takes off[ndim-1-ax]
            for ax in range(ndim):
                q[ax] = p[ax] + off[ndim - 1 - ax]
            for ax in range(ndim):
                (kl, kh), (vl, vh) = pairs[ax]
                if q[ax] < 0 and kl == 1:
                    const = vl
                    break
                if q[ax] >= shape[ax] and kh == 1:
                    const = vh
                    break
            if const is not None:
                b[row] += w * const
                continue
            q = [q[ax] % shape[ax] for ax in range(ndim)]
            M[row, np.ravel_multi_index(tuple(q), shape)] += w
    return M, b


def swe_matrix(shape, dt, g, H):
    """Dense one-step matrix of the C-grid shallow-water update, periodic.

    State vector = [h; u; v], each flattened C-order, shape (ny, nx).
    """
    ny, nx = shape
    n = ny * nx
    M = np.eye(3 * n)

    def idx(j, i):
        return (j % ny) * nx + (i % nx)

    for j in range(ny):
        for i in range(nx):
            p = idx(j, i)
            # h' = h - dt H [(u(i,j) - u(i-1,j)) + (v(i,j) - v(i,j-1))]
            M[p, n + idx(j, i)] += -dt * H
            M[p, n + idx(j, i - 1)] += dt * H
            M[p, 2 * n + idx(j, i)] += -dt * H
            M[p, 2 * n + idx(j - 1, i)] += dt * H
            # u' = u - dt g (h(i+1,j) - h(i,j))
            M[n + p, idx(j, i + 1)] += -dt * g
            M[n + p, idx(j, i)] += dt * g
            # v' = v - dt g (h(i,j+1) - h(i,j))
            M[2 * n + p, idx(j + 1, i)] += -dt * g
            M[2 * n + p, idx(j, i)] += dt * g
    return M


def normwise(a, b):
    """max|a - b| / max|b| (0 when both vanish)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    num = np.max(np.abs(a - b))
    return float(num / den) if den > 0 else float(num)


def read_blocks(path):
    """Read '#'-separated integer blocks of a golden fixture file."""
    blocks, cur = [], []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line:
                continue
            if line.startswith("#"):
                if cur:
                    blocks.append(np.array(cur, dtype=np.float64))
                    cur = []
                continue
            cur.append([float(x) for x in line.split()])
    if cur:
        blocks.append(np.array(cur, dtype=np.float64))
    return blocks
