"""The C ABI without a GPU: the library loads, exports every function include/ssht.h declares,
and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_0807_4494_gb300 import build, ssht
    if not os.path.exists(ssht.LIB_PATH):
        build.build()
    return ssht, ssht._lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ssht.h")).read()
    return re.findall(r"SSHT_API\s+[\w\s\*]+?\b(ssht_\w+)\s*\(", src)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("ssht_plan", "ssht_plan_ex", "ssht_inverse", "ssht_forward", "ssht_adjoint", "ssht_plan_destroy",
                 "ssht_last_error"):
        assert want in names


def test_library_exports_every_declared_function():
    ssht, lib = _lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(ssht.EXPORTS)
    assert ssht.ssht_version() >= 100


@pytest.mark.parametrize("L,s,B,prec,mode", [(0, 0, 1, 0, 0), (2049, 0, 1, 0, 0), (8, 8, 1, 0, 0), (8, -8, 1, 0, 0),
                                             (8, 0, 0, 0, 0), (8, 0, 1, 7, 0), (8, 0, 1, 0, 5)])
def test_invalid_plan_arguments_are_rejected(L, s, B, prec, mode):
    ssht, lib = _lib()
    h = ctypes.c_void_p()
    d = ssht.PlanDesc(L, s, B, prec, mode, 0)
    rc = lib.ssht_plan_ex(ctypes.byref(h), ctypes.byref(d))
    assert rc == -1 and not h.value
    assert len(ssht.ssht_last_error()) > 0


def test_null_arguments_are_rejected():
    ssht, lib = _lib()
    assert lib.ssht_plan_ex(None, None) == -1
    assert lib.ssht_inverse(None, None, None, None) == -1
    assert lib.ssht_forward(None, None, None, None) == -1
    assert lib.ssht_adjoint(None, None, None, None) == -1
    assert lib.ssht_plan_check(None) == -1
    n = ctypes.c_int()
    assert lib.ssht_plan_profile_trace(None, None, None, None, None, 0, ctypes.byref(n)) == -1
    assert lib.ssht_plan_destroy(None) == 0


def test_release_build_checks_no_indices():
    """ssht_debug_bounds answers SSHT_EUNSUPPORTED in a release build (no device call)."""
    ssht, lib = _lib()
    with pytest.raises(ssht.SshtError) as e:
        ssht.ssht_debug_bounds()
    assert e.value.code == -5


def test_bounds_checked_build_compiles_and_exports_the_same_boundary():
    """The library compiled with -DSSHT_DEBUG (the index-checked build its GPU test runs) builds
    here and exports every declared function."""
    from paper_0807_4494_gb300 import build
    lib = ctypes.CDLL(build.build(debug=True))
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_sends_host_data_calls_to_the_current_stream(monkeypatch):
    """The binding passes the calling thread's current CUDA stream for every call, whether the
    data tensor is on the device or on the host (a plan owns one workspace, so an inverse from
    host memory and the forward of its device result must go to one stream in order)."""
    import torch
    from paper_0807_4494_gb300 import ssht

    class FakeStream:
        cuda_stream = 0xBEEF

    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: FakeStream())
    host = torch.zeros(4, dtype=torch.complex64)
    assert ssht.Plan._stream(None, host) == 0xBEEF
    assert ssht.Plan._stream(7, host) == 7
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    assert ssht.Plan._stream(None, host) == 0
