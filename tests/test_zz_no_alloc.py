"""ssht_wigner_delta_noalloc: the Delta table computed without allocating device memory.

Who needs it: callers that cannot call cudaMalloc, e.g. a host application that has reserved
nearly all device memory for its own pool before loading the library, or a latency-critical loop
that must not pay for an allocation and the synchronisation it can cause.  The entry point keeps
its scratch in a fixed array inside the library (band-limits up to 512).

This file is collected last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-13  # the tolerance of the Delta-table parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _lib():
    from paper_0807_4494_gb300 import ssht
    return ssht, ssht._lib()


def _noalloc(L):
    ssht, lib = _lib()
    n = L * (L + 1) * (2 * L + 1) // 6
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.ssht_wigner_delta_noalloc(L, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert rc == 0, ssht.ssht_last_error()
    return out


def _with_plan(L):
    """The same table from the plan entry point, made with the same (Risbo) recursion."""
    ssht, _ = _lib()
    plan = ssht.Plan(L, 0, 1, recursion="risbo")
    ref = plan.wigner_delta()
    plan.check()
    return ref


def test_noalloc_matches_plan_entry_point_on_consecutive_calls():
    L = 512
    first = _noalloc(L)
    second = _noalloc(L)  # the scratch array keeps the first call's contents
    torch.cuda.synchronize()
    ref = _with_plan(L)
    for out in (first, second):
        assert not torch.isnan(out).any()
        assert float((out - ref).abs().max()) < TOL
    small = _noalloc(37)
    torch.cuda.synchronize()
    assert float((small - _with_plan(37)).abs().max()) < TOL


def test_noalloc_rejects_band_limits_beyond_its_scratch():
    ssht, lib = _lib()
    buf = torch.empty(8, dtype=torch.float64, device="cuda")
    for L in (0, 513, 1024):
        rc = lib.ssht_wigner_delta_noalloc(L, ctypes.c_void_p(buf.data_ptr()), None)
        assert rc == -1
        assert "512" in ssht.ssht_last_error() or L == 0
    assert lib.ssht_wigner_delta_noalloc(16, None, None) == -1


def test_noalloc_timeout_marks_the_table_and_the_next_call_recovers():
    """A wait of the recursion that runs out (a 1 ns limit: the first hand-off between CTAs gives
    up) makes the kernel leave and the call's table start with a NaN; the device stays usable and
    the next call, with the default limit, is right again."""
    ssht, _ = _lib()
    L = 64
    ssht.ssht_debug_noalloc_wait_limit(1)
    try:
        bad = _noalloc(L)
        torch.cuda.synchronize()
    finally:
        ssht.ssht_debug_noalloc_wait_limit(0)
    assert torch.isnan(bad[0])
    good = _noalloc(L)
    torch.cuda.synchronize()
    ref = _with_plan(L)
    assert not torch.isnan(good).any()
    assert float((good - ref).abs().max()) < TOL
