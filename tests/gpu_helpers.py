"""Helpers for the GPU parity tests: move seeded inputs to the device in a
storage dtype, read results back as FP64, and the tolerance formulas.

Tolerances (max-abs unless stated), written from the arithmetic:
* FP64 storage: normwise max|gpu - oracle| / max|oracle| <= 1e-12.
* FP32 storage, FP32 arithmetic: each sweep commits at most `nops` roundings of
  relative size 2^-24 on values bounded by M = max|u|, and the per-step
  operator norm G = ||A||_inf carries earlier errors forward, so
  |err_T| <= sum_{t<T} G^t * nops * 2^-24 * M.
* BF16 storage, FP32 arithmetic: every sweep rounds the stored value once to
  bfloat16 (at most half an ulp, relative 2^-8 at 8 significant bits), which
  dominates the FP32 roundings: |err_T| <= sum_{t<T} G^t * (2^-8 + nops*2^-24) * M.
The long full-size runs and the shallow-water and Gray-Scott cases use the
sharper bounds of error_bounds.py instead.
"""
from __future__ import annotations

import numpy as np
import torch

import lope_inputs as LI

TORCH_DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def to_device(x64: np.ndarray, dtype: str):
    """Round an FP64 field to `dtype`; return (device tensor, stored values as FP64)."""
    stored = LI.to_storage(x64, dtype)
    t = torch.from_numpy(np.ascontiguousarray(stored))
    if dtype == "bf16":
        t = t.to(torch.bfloat16)
    return t.to("cuda"), np.asarray(stored, dtype=np.float64)


def to_host(t) -> np.ndarray:
    return t.detach().to(torch.float64).cpu().numpy()


def normwise(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    num = np.max(np.abs(a - b))
    return float(num / den) if den > 0 else float(num)


def bound_f32(nsteps: int, M: float, nops: int = 8, G: float = 1.0) -> float:
    s = sum(G ** t for t in range(nsteps))
    return s * nops * 2.0 ** -24 * M * 1.0001 + 1e-30


def bound_bf16(nsteps: int, M: float, nops: int = 8, G: float = 1.0) -> float:
    s = sum(G ** t for t in range(nsteps))
    return s * (2.0 ** -8 + nops * 2.0 ** -24) * M * 1.0001


def sub_box(shape, center, radius, periodic):
    """Index arrays of the box center +- radius (wrapped on periodic axes,
    clipped on the others) and the position of `center` inside it."""
    idx, pos = [], []
    for ax, (n, c) in enumerate(zip(shape, center)):
        if periodic[ax] and 2 * radius + 1 < n:
            ii = np.arange(c - radius, c + radius + 1) % n
            idx.append(ii)
            pos.append(radius)
        else:
            lo, hi = max(0, c - radius), min(n, c + radius + 1)
            if periodic[ax]:
                lo, hi = 0, n
            idx.append(np.arange(lo, hi))
            pos.append(c - lo)
    return idx, tuple(pos)
