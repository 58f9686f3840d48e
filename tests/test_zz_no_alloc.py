"""The reduction entry point that allocates nothing (lope_reduce_noalloc).

Callers whose device memory belongs entirely to another allocator, or who
cannot afford an allocation call in their loop, use this entry point: its
partial sums live in the library's own static device array.  Its result must
agree with lope_reduce (which takes a scratch buffer) within the tolerance of
the other reduction tests, on two calls in a row (the second call reuses the
array the first one left behind).  This file is collected last on purpose.
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
    return t.cuda()


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
def test_noalloc_reduce_matches_scratch_reduce_twice(lope, dtype):
    L = lope
    stream = torch.cuda.current_stream().cuda_stream
    code = L.DTYPES[dtype]
    for call, (shape, seed) in enumerate((((1000, 777), 12), ((1500, 901), 13))):
        x = _dev(LI.uniform_field(seed, shape), dtype)
        y = _dev(LI.normal_field(seed + 100, shape), dtype)
        n = x.numel()
        for op in (0, 1):
            ref = torch.empty(1, dtype=torch.float64, device="cuda")
            scratch = torch.empty(L.lope_reduce_scratch_bytes(), dtype=torch.uint8, device="cuda")
            L.lope_reduce(op, code, x.data_ptr(), y.data_ptr(), n, ref.data_ptr(),
                          scratch.data_ptr(), stream)
            got = torch.empty(1, dtype=torch.float64, device="cuda")
            L.lope_reduce_noalloc(op, code, x.data_ptr(), y.data_ptr(), n, got.data_ptr(), stream)
            torch.cuda.synchronize()
            a, b = float(got.item()), float(ref.item())
            assert abs(a - b) <= 1e-9 * abs(b), (call, op, a, b)


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
