"""The reduction entry point that allocates nothing (lope_reduce_noalloc).

Callers whose device memory belongs entirely to another allocator, or who
cannot afford an allocation call in their loop, use this entry point: its
partial sums live in the library's own static device array.  Its result must
agree with lope_reduce (which takes a scratch buffer) and with an FP64 sum on
the host, within the tolerance of the other reduction tests, on calls in a row
that go from large to small (each later call sits on partial-sum slots an
earlier, larger call left behind) and on a case near the 2^28-element limit.
This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import lope_inputs as LI

pytestmark = pytest.mark.gpu


def _dev(x64, dtype):
    stored = LI.to_storage(x64, dtype)
    t = torch.from_numpy(np.ascontiguousarray(stored))
    if dtype == "bf16":
        t = t.to(torch.bfloat16)
    return t.cuda(), np.asarray(stored, dtype=np.float64)


def _both(L, op, code, x, y, n, stream):
    ref = torch.empty(1, dtype=torch.float64, device="cuda")
    scratch = torch.empty(L.lope_reduce_scratch_bytes(), dtype=torch.uint8, device="cuda")
    L.lope_reduce(op, code, x.data_ptr(), y.data_ptr(), n, ref.data_ptr(), scratch.data_ptr(),
                  stream)
    got = torch.empty(1, dtype=torch.float64, device="cuda")
    L.lope_reduce_noalloc(op, code, x.data_ptr(), y.data_ptr(), n, got.data_ptr(), stream)
    torch.cuda.synchronize()
    return float(got.item()), float(ref.item())


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
def test_noalloc_reduce_matches_scratch_reduce_large_then_small(lope, dtype):
    L = lope
    stream = torch.cuda.current_stream().cuda_stream
    code = L.DTYPES[dtype]
    # large, then smaller, then a single element: every later call reuses
    # slots an earlier call filled
    for call, (shape, seed) in enumerate((((1500, 901), 13), ((1000, 777), 12), ((1, 1), 14))):
        x, x64 = _dev(LI.uniform_field(seed, shape), dtype)
        y, y64 = _dev(LI.normal_field(seed + 100, shape), dtype)
        n = x.numel()
        for op in (0, 1):
            a, b = _both(L, op, code, x, y, n, stream)
            host = float(np.sum(x64)) if op == 0 else float(np.sum((x64 - y64) ** 2))
            assert abs(a - b) <= 1e-9 * abs(b), (call, op, a, b)
            assert abs(a - host) <= 1e-9 * abs(host), (call, op, a, host)


def test_noalloc_reduce_near_the_size_limit(lope):
    """2^28 - 777 FP32 elements: all 65 536 partial-sum slots but a ragged last
    one; checked against lope_reduce and a host FP64 sum."""
    L = lope
    stream = torch.cuda.current_stream().cuda_stream
    n = (1 << 28) - 777
    x, x64 = _dev(LI.uniform(1400, n), "f32")
    host = float(np.sum(x64))
    del x64
    a, b = _both(L, 0, L.DTYPES["f32"], x, x, n, stream)
    assert abs(a - b) <= 1e-9 * abs(b), (a, b)
    assert abs(a - host) <= 1e-9 * abs(host), (a, host)
    # a small call right after the largest one
    a, b = _both(L, 0, L.DTYPES["f32"], x, x, 5, stream)
    assert abs(a - b) <= 1e-12 * abs(b) and abs(a - float(np.sum(x[:5].double().cpu().numpy()))) <= 1e-12


def test_noalloc_reduce_rejects_oversize_and_handles_empty(lope):
    L = lope
    stream = torch.cuda.current_stream().cuda_stream
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    res = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LopeError, match="2\\^28"):
        L.lope_reduce_noalloc(0, L.DTYPES["f32"], x.data_ptr(), 0, (1 << 28) + 1, res.data_ptr(),
                              stream)
    L.lope_reduce_noalloc(0, L.DTYPES["f32"], x.data_ptr(), 0, 0, res.data_ptr(), stream)
    torch.cuda.synchronize()
    assert float(res.item()) == 0.0
