"""mm_totals_noalloc: the allocation-free totals entry point, for callers that
cannot allocate device memory (stream capture, no implicit synchronisation,
a host-owned memory pool).  It must give the context-based mm_totals result
on consecutive calls, even though every call reuses one static scratch
array, and must reject sizes beyond its limit with a clear error.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def call_noalloc(L, U, totals, n, stream):
    buf = ctypes.create_string_buffer(256)
    st = L.mm_totals_noalloc(ctypes.c_void_p(U.data_ptr()), n, ctypes.c_void_p(totals.data_ptr()),
                             ctypes.c_void_p(stream.cuda_stream), buf, len(buf))
    return st, buf.value.decode()


def test_noalloc_totals_equal_context_totals_on_consecutive_calls():
    import torch
    from paper_1707_05333_gb300 import binding
    from paper_1707_05333_gb300 import build

    build.build()
    L = binding.load()
    ctx = binding.Context()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(1707)
    # two calls in a row with different sizes and data: the second must not
    # see the first call's partial sums
    for n in (3_000_017, 4097):
        U = torch.tensor(rng.normal(size=(5, n)) + np.array([[3.0], [0.0], [0.0], [0.0], [5.0]]),
                         dtype=torch.float64, device="cuda")
        ref = ctx.mm_totals(U).cpu().numpy()
        got = torch.full((5,), np.nan, dtype=torch.float64, device="cuda")
        st, msg = call_noalloc(L, U, got, n, stream)
        assert st == 0, msg
        got = got.cpu().numpy()
        scale = U.abs().sum(1).cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-13 * scale), (got, ref)
        exact = U.cpu().numpy().sum(1)
        assert np.all(np.abs(got - exact) <= 1e-12 * scale)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1707_05333_gb300 import binding

    L = binding.load()
    stream = torch.cuda.current_stream()
    U = torch.zeros((5, 8), dtype=torch.float64, device="cuda")
    out = torch.zeros((5,), dtype=torch.float64, device="cuda")
    too_many = 16777216 + 1
    st, msg = call_noalloc(L, U, out, too_many, stream)
    assert st == 3 and "exceeds the static scratch limit" in msg
    st, msg = call_noalloc(L, U, out, 0, stream)
    assert st == 1 and msg
