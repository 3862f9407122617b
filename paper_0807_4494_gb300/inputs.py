"""Seeded synthetic inputs for the spin spherical harmonic transform.

This module only draws random numbers into the coefficient layout; it holds none
of the transform's arithmetic.  It is the one module shared by the tests, the
benchmark and the checks of the CUDA path against the CPU oracle.

Layout: coefficients ``flm[b, l*l + l + m]`` (complex) for 0 <= l < L, |m| <= l,
zero for l < |s| (no spin-s harmonic exists there).

Spectra:
  ``"flat"``  Re and Im iid N(0, 1) for every (l, m) with |s| <= l < L;
  ``"cmb"``   complex normal CN(0, 1/(l+1)^2): Re and Im iid N(0, 1/(2 (l+1)^2))
              (a decaying, CMB-like angular power spectrum);
  ``"paper"`` Re and Im iid U[-1, 1] (the test functions of Sec. 4 of the paper);
              with ``real=True`` (s = 0 only) the reality condition
              f_{l,-m} = (-1)^m conj(f_{lm}) is imposed and f_{l0} is real.
Field b of a batch uses ``numpy.random.default_rng(seed + b)``.
"""
import numpy as np


def coeffs(L, s=0, batch=1, seed=0, spectrum="flat", real=False, dtype=np.complex128):
    out = np.zeros((batch, L * L), dtype=np.complex128)
    l = np.repeat(np.arange(L), 2 * np.arange(L) + 1)
    m = np.concatenate([np.arange(-k, k + 1) for k in range(L)]) if L > 0 else np.zeros(0, int)
    valid = l >= abs(s)
    for b in range(batch):
        rng = np.random.default_rng(seed + b)
        if spectrum == "flat":
            re = rng.standard_normal(L * L)
            im = rng.standard_normal(L * L)
        elif spectrum == "cmb":
            sd = 1.0 / (np.sqrt(2.0) * (l + 1.0))
            re = rng.standard_normal(L * L) * sd
            im = rng.standard_normal(L * L) * sd
        elif spectrum == "paper":
            re = rng.uniform(-1.0, 1.0, L * L)
            im = rng.uniform(-1.0, 1.0, L * L)
        else:
            raise ValueError(spectrum)
        x = np.where(valid, re + 1j * im, 0.0)
        if real:
            if s != 0:
                raise ValueError("the reality condition applies to s = 0")
            for k in range(L):
                base = k * k + k
                x[base] = x[base].real
                for mm in range(1, k + 1):
                    x[base - mm] = (-1) ** mm * np.conj(x[base + mm])
        out[b] = x
    return out.astype(dtype)


def uneven_batch(n_fields=256, Ls=(128, 256, 512, 1024), spins=(0, 1, -1, 2, -2), seed=0):
    """Band-limits and spins of an uneven batch: L and s drawn uniformly (one generator)."""
    rng = np.random.default_rng(seed)
    L = rng.choice(np.asarray(Ls), size=n_fields)
    s = rng.choice(np.asarray(spins), size=n_fields)
    return [int(x) for x in L], [int(x) for x in s]
