"""Build and load the oracle's C library (ssht_oracle.c) through ctypes.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ssht_oracle.c")
_SO = os.path.join(_HERE, "libssht_oracle.so")
_lib = None


def build(force=False):
    """Compile ssht_oracle.c with gcc (-O2, no FMA contraction, OpenMP)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", _SO + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        for name, args in [
            ("oracle_wigner_full", [ctypes.c_int, ctypes.c_double, dp]),
            ("oracle_delta_quadrant", [ctypes.c_int, ctypes.c_double, dp]),
            ("oracle_fourier_coeff", [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]),
            ("oracle_harmonic_project", [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]),
            ("oracle_weight_conv", [ctypes.c_int, ctypes.c_int, dp, dp]),
            ("oracle_triangular_forward", [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]),
            ("oracle_triangular_matrix", [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]),
            ("oracle_num_threads", []),
        ]:
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
    return _lib


def ptr(a):
    """Pointer to a C-contiguous float64 (or complex128 viewed as pairs) array."""
    assert a.flags["C_CONTIGUOUS"]
    assert a.dtype in (np.float64, np.complex128)
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")
