"""The product of a double and a small integer by integer operations (csrc/int_mul.h), compiled
for the host from the same header the recursions include, against IEEE multiplication as numpy
performs it (round to nearest, ties to even): random coefficients over the range the recursions
take (a(m') in (1/(2L), 1]) and beyond it, every integer k < 2^11, the power-of-two factor d, and
the boundary cases -- ties (odd significands times 3, 1025 and 2047 round off an exact half),
carries out of 53 bits into the exponent (an all-ones significand), k = 1, powers of two, zero."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_0807_4494_gb300", "csrc", "int_mul.h")

SHIM = r'''
#include "%s"
extern "C" void mul(const unsigned long long* x, const unsigned int* k, int d, unsigned long long* out, long n) {
  for (long i = 0; i < n; ++i) out[i] = ssht::mul_small_rn_bits(x[i], k[i], d);
}
'''


@pytest.fixture(scope="module")
def mul():
    d = tempfile.mkdtemp()
    src = os.path.join(d, "shim.cpp")
    so = os.path.join(d, "shim.so")
    open(src, "w").write(SHIM % HDR)
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", so, src], check=True)
    lib = ctypes.CDLL(so)
    lib.mul.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_long]

    def run(x, k, dd):
        x = np.ascontiguousarray(x, dtype=np.float64)
        k = np.ascontiguousarray(np.broadcast_to(k, x.shape), dtype=np.uint32)
        out = np.empty(x.shape, dtype=np.uint64)
        lib.mul(x.ctypes.data, k.ctypes.data, dd, out.ctypes.data, x.size)
        return out
    return run


def ieee(x, k, d):
    return (np.asarray(x, dtype=np.float64) * np.asarray(k, dtype=np.float64) * 2.0 ** d).view(np.uint64)


@pytest.mark.parametrize("d", [0, 1])
def test_random_coefficients(mul, d):
    rng = np.random.default_rng(d)
    for lo, hi in [(-13, 0), (-60, 8), (-1000, 1000)]:
        x = np.exp2(rng.uniform(lo, hi, 400000))
        k = rng.integers(0, 2048, x.size)
        assert np.array_equal(mul(x, k, d), ieee(x, k, d))
    # random significand bit patterns (all 52 fraction bits live)
    bits = rng.integers(0, 2 ** 52, 400000, dtype=np.uint64)
    x = ((np.uint64(1013) << np.uint64(52)) | bits).view(np.float64)
    k = rng.integers(0, 2048, x.size)
    assert np.array_equal(mul(x, k, d), ieee(x, k, d))


def test_every_k(mul):
    rng = np.random.default_rng(7)
    x = np.exp2(rng.uniform(-12, 0, 256))
    for k in range(2048):
        assert np.array_equal(mul(x, k, 1), ieee(x, k, 1)), k


def test_ties_and_carries(mul):
    rng = np.random.default_rng(3)
    frac = rng.integers(0, 2 ** 52, 200000, dtype=np.uint64) | np.uint64(1)  # odd significands
    x = ((np.uint64(1020) << np.uint64(52)) | frac).view(np.float64)
    for k in (3, 5, 1025, 2047):
        got, want = mul(x, k, 0), ieee(x, k, 0)
        assert np.array_equal(got, want), k
    ones = np.array([((1020 << 52) | (2 ** 52 - 1))], dtype=np.uint64).view(np.float64)
    for k in range(1, 2048):
        assert np.array_equal(mul(ones, k, 0), ieee(ones, k, 0)), k
    special = np.array([0.0, 1.0, 0.5, 2.0 ** -30, 1 - 2 ** -53, 1 + 2 ** -52], dtype=np.float64)
    for k in (0, 1, 2, 1024, 2047):
        assert np.array_equal(mul(special, k, 1), ieee(special, k, 1)), k
