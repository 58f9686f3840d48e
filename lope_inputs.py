"""Seeded synthetic inputs for the LOPe stencil workloads.

This module is shared by the FP64 oracle (``oracle/``) and by the CUDA path's
tests and benchmark.  It holds only random-number generation and rounding to a
storage dtype; none of the stencil arithmetic lives here.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in counter mode: element ``i`` of the
stream with seed ``s`` is ``mix(s + (i + 1) * 0x9E3779B97F4A7C15)``, where
``mix`` is the SplitMix64 output function.  A uniform double in [0, 1) takes the
top 53 bits.  Normals use the Box-Muller transform on the uniform pair at
counters (2i, 2i + 1).

Seeds: workload ``i`` of the benchmark table uses seed ``1000 + i`` for its
fields and ``2000 + i`` for a target field.  Several fields of one grid take
consecutive, non-overlapping counter ranges of the same seed, in field order.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise (uint64, wrapping)."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Raw 64-bit outputs ``offset .. offset+n-1`` of the counter-mode stream."""
    out = np.empty(n, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for a in range(0, n, _CHUNK):
            b = min(n, a + _CHUNK)
            ctr = np.arange(offset + a + 1, offset + b + 1, dtype=np.uint64)
            out[a:b] = _mix(s + ctr * _GOLDEN)
    return out


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each output."""
    out = np.empty(n, dtype=np.float64)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        r = splitmix64(seed, b - a, offset + a)
        out[a:b] = (r >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return out


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller on uniforms (2i, 2i+1) past ``2*offset``."""
    out = np.empty(n, dtype=np.float64)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        u = uniform(seed, 2 * (b - a), 2 * (offset + a))
        u1, u2 = u[0::2], u[1::2]
        out[a:b] = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    return out


def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round doubles to the nearest bfloat16 (ties to even); result as float32.

    The rounding is done once, on the binary64 pattern (7 kept fraction bits),
    so there is no double rounding through binary32.  Inputs are finite and far
    from the bfloat16 overflow threshold.
    """
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    keep = np.uint64(45)  # 52 - 7 fraction bits dropped
    with np.errstate(over="ignore"):
        lsb = (b >> keep) & np.uint64(1)
        b = (b + (np.uint64((1 << 44) - 1) + lsb)) & ~np.uint64((1 << 45) - 1)
    return b.view(np.float64).astype(np.float32)


def to_storage(x: np.ndarray, dtype: str) -> np.ndarray:
    """Round an FP64 field to the storage dtype; returns the stored values.

    ``dtype`` is "f64", "f32" or "bf16".  For "bf16" the returned float32 array
    holds exactly the bfloat16 values.
    """
    if dtype == "f64":
        return np.asarray(x, dtype=np.float64).copy()
    if dtype == "f32":
        return np.asarray(x, dtype=np.float64).astype(np.float32)
    if dtype == "bf16":
        return round_to_bf16(x)
    raise ValueError(f"unknown storage dtype {dtype!r}")


def uniform_field(seed: int, shape, offset: int = 0) -> np.ndarray:
    """U[0,1) field of the given shape (C order: last axis fastest)."""
    n = int(np.prod(shape))
    return uniform(seed, n, offset).reshape(shape)


def normal_field(seed: int, shape, offset: int = 0) -> np.ndarray:
    n = int(np.prod(shape))
    return normal(seed, n, offset).reshape(shape)


def swe_fields(seed: int, shape):
    """(h, u, v) initial state of the shallow-water workload.

    h = 1 + 0.01 N(0,1), u = 0.1 N(0,1), v = 0.1 N(0,1); the three fields take
    consecutive counter ranges of one seed, in the order h, u, v.
    """
    n = int(np.prod(shape))
    h = 1.0 + 0.01 * normal(seed, n, 0).reshape(shape)
    u = 0.1 * normal(seed, n, n).reshape(shape)
    v = 0.1 * normal(seed, n, 2 * n).reshape(shape)
    return h, u, v


def batch_shapes(seed: int, count: int, lo: int = 64, hi: int = 2048):
    """Grid shapes and boundary kinds of the batched workload.

    Each grid draws ny then nx uniformly from the integers lo..hi inclusive and
    a boundary kind (0 periodic, 1 Dirichlet) with probability 1/2, from
    consecutive uniforms of the seed's stream (three per grid).
    """
    u = uniform(seed, 3 * count, 0)
    span = hi - lo + 1
    shapes, kinds = [], []
    for g in range(count):
        ny = lo + min(span - 1, int(u[3 * g] * span))
        nx = lo + min(span - 1, int(u[3 * g + 1] * span))
        shapes.append((ny, nx))
        kinds.append(0 if u[3 * g + 2] < 0.5 else 1)
    return shapes, kinds
