"""Plain definitions used to pin the oracle (no recursion, no torus, no FFT).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``wigner_d_half_pi_exact``: Wigner's explicit sum for d^j_{m'm}(beta) at beta = pi/2, where every
  term carries (1/sqrt 2)^{2j}; the sum is taken in exact rational arithmetic and one square root
  is taken at the end with 200-bit integer arithmetic.  Works for integer and half-integer j.
* ``wigner_d_sum``: the same explicit sum at any beta in floating point (small j only).
* ``wigner_d_jacobi``: eqn wignerd_b (Jacobi polynomial form) with the symmetry relations used to
  bring the indices to the form the equation needs (second index n >= |m|).
* ``spin_sh`` (eqn ssh_wigner) and ``spin_sh_goldberg`` (eqn ssh_goldberg as printed).
* ``synthesis_direct``: f(theta, phi) = sum_{l,m} sf_lm sY_lm(theta, phi) (eqn ssht_inv).
* ``gauss_legendre_analysis``: sf_lm = int f conj(sY_lm) dOmega (eqn ssht_fwd) by Gauss-Legendre
  quadrature in cos(theta) and the trapezoid rule in phi, exact for band-limited f.
"""
from fractions import Fraction
from math import factorial, isqrt

import numpy as np
from scipy.special import eval_jacobi, gammaln


def wigner_d_half_pi_exact(tj, ta, tb):
    """d^j_{a b}(pi/2) with j = tj/2, a = ta/2 (row), b = tb/2 (column), all doubled integers."""
    assert (tj - ta) % 2 == 0 and (tj - tb) % 2 == 0
    if abs(ta) > tj or abs(tb) > tj:
        return 0.0
    # integer quantities j+a, j-a, j+b, j-b
    jpa, jma, jpb, jmb = (tj + ta) // 2, (tj - ta) // 2, (tj + tb) // 2, (tj - tb) // 2
    amb = (ta - tb) // 2  # a - b, an integer
    S = Fraction(0)
    for k in range(0, tj + 1):
        d1, d2, d3 = jpb - k, amb + k, jma - k
        if d1 < 0 or d2 < 0 or d3 < 0:
            continue
        S += Fraction((-1) ** ((amb + k) % 2), factorial(d1) * factorial(k) * factorial(d2) * factorial(d3))
    if S == 0:
        return 0.0
    P = factorial(jpa) * factorial(jma) * factorial(jpb) * factorial(jmb)
    sq = P * S * S / Fraction(2 ** tj)  # value^2, exact
    bits = 200
    root = isqrt(sq.numerator * (1 << (2 * bits)) // sq.denominator)
    return (1.0 if S > 0 else -1.0) * (root / float(1 << bits))


def wigner_d_sum(tj, ta, tb, beta):
    """Wigner's explicit sum for d^j_{ab}(beta) in double precision (fine for j <~ 10)."""
    jpa, jma, jpb, jmb = (tj + ta) // 2, (tj - ta) // 2, (tj + tb) // 2, (tj - tb) // 2
    amb = (ta - tb) // 2
    c, s = np.cos(beta / 2.0), np.sin(beta / 2.0)
    pref = np.sqrt(float(factorial(jpa) * factorial(jma) * factorial(jpb) * factorial(jmb)))
    tot = 0.0
    for k in range(0, tj + 1):
        d1, d2, d3 = jpb - k, amb + k, jma - k
        if d1 < 0 or d2 < 0 or d3 < 0:
            continue
        ec = tj + (tb - ta) // 2 - 2 * k                  # 2j + b - a - 2k
        es = (ta - tb) // 2 + 2 * k                       # a - b + 2k
        tot += (-1) ** ((amb + k) % 2) * c ** ec * s ** es / (
            factorial(d1) * factorial(k) * factorial(d2) * factorial(d3))
    return pref * tot


def _d_jacobi_core(l, m, n, beta):
    """Eqn wignerd_b for n >= |m| (log-space prefactor)."""
    assert n >= abs(m)
    x = np.cos(beta)
    lf = 0.5 * (gammaln(l + n + 1) + gammaln(l - n + 1) - gammaln(l + m + 1) - gammaln(l - m + 1))
    s2, c2 = np.sin(beta / 2.0), np.cos(beta / 2.0)
    with np.errstate(divide="ignore"):
        ls = np.zeros_like(x) if n == m else (n - m) * np.log(np.abs(s2))
        lc = np.zeros_like(x) if n == -m else (n + m) * np.log(np.abs(c2))
    lp = lf + ls + lc
    sign = np.sign(s2) ** (n - m) * np.sign(c2) ** (n + m)
    val = np.exp(lp) * sign * eval_jacobi(l - n, n - m, n + m, x)
    return np.where(np.isfinite(lp), val, 0.0)


def wigner_d_jacobi(l, m, n, beta):
    """Eqn wignerd_b, with d_{mn} = (-1)^{m-n} d_{nm} (from eqn wignerd_sym3 and D(R^-1) = D(R)^T)
    and eqn wignerd_sym1 used to move the indices into the n >= |m| form."""
    beta = np.asarray(beta, dtype=float)
    if n >= abs(m):
        return _d_jacobi_core(l, m, n, beta)
    if m >= abs(n):
        return (-1.0) ** ((m - n) % 2) * _d_jacobi_core(l, n, m, beta)
    if -n >= abs(m):
        return (-1.0) ** ((m - n) % 2) * _d_jacobi_core(l, -m, -n, beta)
    return _d_jacobi_core(l, -n, -m, beta)


def spin_sh(l, m, s, theta, phi):
    """Eqn ssh_wigner: sY_lm = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi}."""
    return ((-1.0) ** (s % 2) * np.sqrt((2 * l + 1) / (4 * np.pi)) * wigner_d_jacobi(l, m, -s, theta)
            * np.exp(1j * m * np.asarray(phi)))


def spin_sh_goldberg(l, m, s, theta, phi):
    """Eqn ssh_goldberg exactly as printed (sum over r with non-negative factorial arguments)."""
    theta = np.asarray(theta, dtype=float)
    pref = np.sqrt((2 * l + 1) / (4 * np.pi) * factorial(l + m) * factorial(l - m)
                   / (factorial(l + s) * factorial(l - s)))
    cot = np.cos(theta / 2) / np.sin(theta / 2)
    tot = np.zeros_like(theta)
    for r in range(0, 2 * l + 2):
        a, b = l - s, s - m + r
        if r > a or b < 0 or b > l + s:
            continue
        tot = tot + (factorial(a) // (factorial(r) * factorial(a - r))) * (
            factorial(l + s) // (factorial(b) * factorial(l + s - b))) * (-1.0) ** ((l - s - r) % 2) * cot ** (s - m + 2 * r)
    return pref * np.sin(theta / 2) ** (2 * l) * tot * np.exp(1j * m * np.asarray(phi))


def synthesis_direct(flm, L, s, theta, phi):
    """Eqn ssht_inv: f(theta_i, phi_j) = sum_{l<L} sum_{|m|<=l} sf_lm sY_lm, on the product grid."""
    flm = np.asarray(flm)
    theta = np.asarray(theta, dtype=float)
    phi = np.asarray(phi, dtype=float)
    g = np.zeros((len(theta), 2 * L - 1), dtype=np.complex128)  # g[i, m + L - 1]
    for l in range(abs(s), L):
        cl = (-1.0) ** (s % 2) * np.sqrt((2 * l + 1) / (4 * np.pi))
        for m in range(-l, l + 1):
            g[:, m + L - 1] += flm[l * l + l + m] * cl * wigner_d_jacobi(l, m, -s, theta)
    ms = np.arange(-(L - 1), L)
    return g @ np.exp(1j * np.outer(ms, phi))


def gauss_legendre_analysis(f_func, L, s, nq=None):
    """Eqn ssht_fwd by quadrature: Gauss-Legendre in cos(theta) with nq >= L nodes (exact to degree
    2nq - 1 >= 2L - 2, the degree of f conj(sY) in cos(theta)) and 2L - 1 equispaced phi (exact for
    phi frequencies |k| <= 2L - 2).  ``f_func(theta, phi)`` returns f on the product grid."""
    nq = nq or L
    x, w = np.polynomial.legendre.leggauss(nq)
    theta = np.arccos(x)
    nphi = 2 * L - 1
    phi = 2 * np.pi * np.arange(nphi) / nphi
    f = f_func(theta, phi)                      # [nq, nphi]
    ms = np.arange(-(L - 1), L)
    fm = f @ np.exp(-1j * np.outer(phi, ms)) * (2 * np.pi / nphi)   # [nq, m]
    flm = np.zeros(L * L, dtype=np.complex128)
    for l in range(abs(s), L):
        cl = (-1.0) ** (s % 2) * np.sqrt((2 * l + 1) / (4 * np.pi))
        for m in range(-l, l + 1):
            flm[l * l + l + m] = np.sum(w * fm[:, m + L - 1] * cl * wigner_d_jacobi(l, m, -s, theta))
    return flm
