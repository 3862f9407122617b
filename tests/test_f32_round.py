"""The FP64 -> FP32 rounding by integer operations (csrc/f32_round.h), compiled for the host from
the same header the kernels include, against IEEE round-to-nearest-even as numpy applies it
(the rounding __double2float_rn performs): random doubles over the whole range the operands take
(normal FP32 range, the FP32 subnormal range and below it), and the boundary cases -- ties,
carries into the exponent, the smallest normal and subnormal, 2^-150 and just above it."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_0807_4494_gb300", "csrc", "f32_round.h")

SHIM = r'''
#include "%s"
extern "C" void convert(const unsigned long long* in, unsigned int* out, long n) {
  for (long i = 0; i < n; ++i) out[i] = ssht::f64_bits_to_f32_rn(in[i]);
}
'''


@pytest.fixture(scope="module")
def convert():
    d = tempfile.mkdtemp()
    src = os.path.join(d, "shim.cpp")
    so = os.path.join(d, "shim.so")
    open(src, "w").write(SHIM % HDR)
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", so, src], check=True)
    lib = ctypes.CDLL(so)
    lib.convert.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long]

    def run(x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.empty(x.shape, dtype=np.uint32)
        lib.convert(x.ctypes.data, out.ctypes.data, x.size)
        return out
    return run


def ieee(x):
    with np.errstate(over="ignore", under="ignore"):
        return np.asarray(x, dtype=np.float64).astype(np.float32).view(np.uint32)


def test_random_doubles_over_the_operand_range(convert):
    rng = np.random.default_rng(0)
    for lo, hi in [(-126, 4), (-150, -126), (-160, -148), (-1074, -150)]:
        e = rng.uniform(lo, hi, 200000)
        x = np.exp2(e) * rng.choice([-1.0, 1.0], e.size)
        assert np.array_equal(convert(x), ieee(x))
    # random bit patterns of doubles with exponents in the same window
    bits = rng.integers(0, 2 ** 52, 200000, dtype=np.uint64)
    ef = rng.integers(1023 - 160, 1023 + 4, 200000).astype(np.uint64)
    x = ((ef << np.uint64(52)) | bits).view(np.float64)
    assert np.array_equal(convert(x), ieee(x))


def test_boundary_cases(convert):
    f32 = np.float32
    tiny = float(np.finfo(f32).tiny)           # 2^-126
    sub = float(np.finfo(f32).smallest_subnormal)  # 2^-149
    cases = [0.0, -0.0, 1.0, -1.0, tiny, -tiny, sub, -sub, sub / 2, sub / 2 * (1 + 2 ** -52),
             sub * 1.5, sub * 2.5, tiny * (1 - 2 ** -24), tiny * (1 - 2 ** -25), tiny * (1 - 2 ** -30),
             1 + 2 ** -24, 1 + 3 * 2 ** -24, 1 + 2 ** -24 + 2 ** -52, 2 - 2 ** -25, 3.0 - 2 ** -24,
             np.nextafter(tiny, 0), np.nextafter(sub, 0), 2.0 ** -1074, 2.0 ** -1023, 13.5, -19.99]
    x = np.array(cases, dtype=np.float64)
    assert np.array_equal(convert(x), ieee(x))
