"""Pins of the oracle's transforms against definitions outside the method.

* inverse: direct synthesis sum_{lm} sf_lm sY_lm with sY from scipy (s = 0), from eqn ssh_wigner
  with eqn wignerd_b (any s) and from eqn ssh_goldberg (times (-1)^m);
* forward: independent Gauss-Legendre quadrature of eqn ssht_fwd; left inverse of the dense
  synthesis matrix; roundtrip on band-limited coefficients;
* adjoint: dot-product test and the conjugate transpose of the dense synthesis matrix;
* the weight w(p) against numerical integration;
* the torus symmetry eqn Ffourier_sym;
* Parseval: the sphere integral of |f|^2 of the direct synthesis equals sum |sf_lm|^2;
* the paper's triangular forward: its printed L = 5 sparsity pattern, machine precision at small
  band-limits and error growth with the band-limit (Sec. 4.2).
"""
import os

import numpy as np
import pytest

from oracle import brute
from oracle import transforms as T
from paper_0807_4494_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def test_spin0_harmonics_equal_scipy():
    from scipy.special import sph_harm_y
    th = np.linspace(0.05, np.pi, 9)
    ph = np.linspace(0.0, 6.0, 9)
    for l in range(0, 12):
        for m in range(-l, l + 1):
            assert np.abs(brute.spin_sh(l, m, 0, th, ph) - sph_harm_y(l, m, th, ph)).max() < 1e-13


def test_goldberg_form_is_wigner_form_times_minus_one_to_m():
    """Reading of eqn ssh_goldberg: as printed it equals (-1)^m times eqn ssh_wigner."""
    th = np.linspace(0.1, 3.0, 11)
    for l in range(0, 8):
        for s in range(-l, l + 1):
            for m in range(-l, l + 1):
                a = brute.spin_sh(l, m, s, th, 0.7)
                g = brute.spin_sh_goldberg(l, m, s, th, 0.7)
                assert np.abs(a - (-1.0) ** (m % 2) * g).max() < 1e-12, (l, m, s)


@pytest.mark.parametrize("L,s", [(1, 0), (2, 0), (7, 0), (16, 0), (8, 2), (9, -1), (13, 3), (16, -2), (24, 2)])
def test_inverse_equals_direct_synthesis(L, s):
    flm = inputs.coeffs(L, s, 1, seed=3)[0]
    f = T.inverse(flm, L, s)
    fd = brute.synthesis_direct(flm, L, s, T.thetas(L), T.phis(L))
    assert f.shape == (L, 2 * L - 1)
    assert rel(f, fd) < 1e-13


def test_inverse_s0_against_scipy_synthesis():
    from scipy.special import sph_harm_y
    L = 10
    flm = inputs.coeffs(L, 0, 1, seed=11)[0]
    th, ph = np.meshgrid(T.thetas(L), T.phis(L), indexing="ij")
    fd = np.zeros_like(th, dtype=complex)
    for l in range(L):
        for m in range(-l, l + 1):
            fd += flm[l * l + l + m] * sph_harm_y(l, m, th, ph)
    assert rel(T.inverse(flm, L, 0), fd) < 1e-13


def test_inverse_against_goldberg_synthesis():
    L, s = 8, 2
    flm = inputs.coeffs(L, s, 1, seed=4)[0]
    th, ph = np.meshgrid(T.thetas(L)[:-1], T.phis(L), indexing="ij")  # cot(theta/2) needs theta < pi
    fd = np.zeros_like(th, dtype=complex)
    for l in range(abs(s), L):
        for m in range(-l, l + 1):
            fd += flm[l * l + l + m] * (-1.0) ** (m % 2) * brute.spin_sh_goldberg(l, m, s, th, ph)
    assert rel(T.inverse(flm, L, s)[:-1], fd) < 1e-12


@pytest.mark.parametrize("L,s", [(6, 0), (11, 1), (14, -2)])
def test_fourier_coeff_symmetry(L, s):
    """Eqn Ffourier_sym: F_{m,-m'} = (-1)^{m+s} F_{m m'} (the oracle computes every m' directly)."""
    flm = inputs.coeffs(L, s, 1, seed=2)[0]
    F = T.fourier_coeff(flm, L, s)
    Lp = L - 1
    for m in range(-Lp, Lp + 1):
        sgn = (-1.0) ** ((m + s) % 2)
        assert np.abs(F[m + Lp, ::-1] - sgn * F[m + Lp, :]).max() < 1e-13 * np.abs(F).max()


def test_weight_against_numerical_integration():
    """w(p) = int_0^pi sin(theta) e^{i p theta} d theta, through the oracle's convolution of a unit impulse."""
    from scipy.integrate import quad
    L = 6
    Lp, N = L - 1, 2 * L - 1
    for mpp in (-3, 0, 2):
        F = np.zeros((N, N), dtype=complex)
        F[0, mpp + Lp] = 1.0
        G = T.weight_conv(F, L)
        for mp in range(-Lp, Lp + 1):
            p = mpp - mp
            re = quad(lambda t: np.sin(t) * np.cos(p * t), 0, np.pi)[0]
            im = quad(lambda t: np.sin(t) * np.sin(p * t), 0, np.pi)[0]
            assert abs(G[0, mp + Lp] - 2 * np.pi * (re + 1j * im)) < 1e-12


@pytest.mark.parametrize("L,s", [(6, 0), (9, 2), (12, -1)])
def test_gauss_legendre_quadrature_recovers_coefficients(L, s):
    """Pins the direct-synthesis and quadrature machinery: eqn ssht_fwd by Gauss-Legendre."""
    flm = inputs.coeffs(L, s, 1, seed=9)[0]
    got = brute.gauss_legendre_analysis(lambda th, ph: brute.synthesis_direct(flm, L, s, th, ph), L, s)
    assert rel(got, flm) < 1e-13


@pytest.mark.parametrize("L,s", [(5, 0), (8, 2), (9, -1), (12, 3)])
def test_parseval_of_direct_synthesis(L, s):
    """Orthonormal spin harmonics: the integral of |f|^2 over the sphere is sum |sf_lm|^2.
    |f|^2 is a polynomial of degree <= 2L - 2 in cos(theta) (the half-angle powers of d^l_{m,-s}
    pair up for equal m and s) with phi frequencies |k| <= 2L - 2, so Gauss-Legendre with L nodes
    and 4L uniform phi points integrate it exactly."""
    flm = inputs.coeffs(L, s, 1, seed=11)[0]
    x, w = np.polynomial.legendre.leggauss(L)
    nphi = 4 * L
    phi = 2 * np.pi * np.arange(nphi) / nphi
    f = brute.synthesis_direct(flm, L, s, np.arccos(x), phi)
    integral = float(np.sum(w[:, None] * np.abs(f) ** 2) * 2 * np.pi / nphi)
    norm2 = float(np.sum(np.abs(flm) ** 2))
    assert abs(integral - norm2) < 1e-12 * norm2


@pytest.mark.parametrize("L,s", [(1, 0), (2, 1), (5, 0), (10, 2), (17, -3), (24, 0)])
def test_forward_on_directly_synthesised_samples(L, s):
    """The oracle forward applied to samples from the definition (not from the oracle's inverse)."""
    flm = inputs.coeffs(L, s, 1, seed=5)[0]
    f = brute.synthesis_direct(flm, L, s, T.thetas(L), T.phis(L))
    assert rel(T.forward(f, L, s), flm) < 1e-13


def synthesis_matrix(L, s):
    """Dense matrix of eqn ssht_inv on the sampling grid: columns = unit coefficients."""
    cols = []
    th, ph = T.thetas(L), T.phis(L)
    for idx in range(L * L):
        e = np.zeros(L * L, dtype=complex)
        e[idx] = 1.0
        cols.append(brute.synthesis_direct(e, L, s, th, ph).ravel())
    return np.array(cols).T


@pytest.mark.parametrize("L,s", [(4, 0), (5, 1), (6, -2)])
def test_forward_is_left_inverse_of_dense_synthesis(L, s):
    A = synthesis_matrix(L, s)
    lo = s * s  # coefficients with l < |s| do not exist
    X = np.stack([T.forward(A[:, k].reshape(L, 2 * L - 1), L, s) for k in range(L * L)], axis=1)
    eye = np.eye(L * L)
    eye[:lo, :lo] = 0.0
    assert np.abs(X - eye).max() < 1e-13


@pytest.mark.parametrize("L,s", [(4, 0), (5, 1), (6, -2)])
def test_adjoint_is_conjugate_transpose_of_synthesis(L, s):
    A = synthesis_matrix(L, s)
    g = np.random.default_rng(1).standard_normal(A.shape[0]) + 1j * np.random.default_rng(2).standard_normal(A.shape[0])
    want = A.conj().T @ g
    got = T.adjoint(g.reshape(L, 2 * L - 1), L, s)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("L,s", [(16, 0), (33, 2), (64, -1)])
def test_adjoint_dot_product(L, s):
    a = inputs.coeffs(L, s, 1, seed=6)[0]
    rng = np.random.default_rng(7)
    g = rng.standard_normal((L, 2 * L - 1)) + 1j * rng.standard_normal((L, 2 * L - 1))
    lhs = np.vdot(T.inverse(a, L, s), g)
    rhs = np.vdot(a, T.adjoint(g, L, s))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("L,s,spectrum", [(64, 2, "flat"), (128, 0, "flat"), (128, 2, "cmb"), (100, -1, "flat")])
def test_roundtrip_forward_inverse_identity(L, s, spectrum):
    flm = inputs.coeffs(L, s, 2, seed=0, spectrum=spectrum)
    back = T.forward(T.inverse(flm, L, s), L, s)
    assert rel(back, flm) < 1e-13


def test_batch_is_fieldwise():
    L, s = 12, 1
    flm = inputs.coeffs(L, s, 3, seed=20)
    f = T.inverse(flm, L, s)
    for b in range(3):
        assert np.array_equal(f[b], T.inverse(flm[b], L, s))


def test_triangular_pattern_matches_paper_example():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "triangular_s0_L5_pattern.txt")) if ln.strip() and not ln.startswith("#")]
    want = np.array([[c == "*" for c in r] for r in rows])
    D = T.triangular_matrix(6, 0, 0)
    assert np.array_equal(np.abs(D) > 1e-12, want)


def test_triangular_forward_small_band_limit_is_exact():
    """Sec. 4.2: for very low band-limits the errors are of the order of machine precision."""
    for L, s in ((4, 0), (8, 0), (9, 2)):
        flm = inputs.coeffs(L, s, 1, seed=1, spectrum="paper")[0]
        back = T.forward_triangular(T.inverse(flm, L, s), L, s)
        assert np.abs(back - flm).max() < 1e-11


def test_triangular_forward_error_grows_with_band_limit():
    """Sec. 4.2: the paper's forward is unstable, its error growing quickly with the band-limit,
    while the quadrature forward stays at machine precision."""
    errs, qerrs = [], []
    for L in (9, 17, 33, 65):
        flm = inputs.coeffs(L, 0, 1, seed=2, spectrum="paper", real=True)[0]
        f = T.inverse(flm, L, 0)
        errs.append(np.abs(T.forward_triangular(f, L, 0) - flm).max())
        qerrs.append(np.abs(T.forward(f, L, 0) - flm).max())
    assert errs[-1] > 1e3 * errs[0]
    assert max(qerrs) < 1e-12


def test_triangular_conditioning_is_extreme():
    """Sec. 4.2 quotes cond = 6e14 for 0D_38 at band-limit 50; the square block of rows and
    columns >= 38 is at least that badly conditioned here (order of magnitude only)."""
    D = T.triangular_matrix(51, 0, 38)
    assert np.linalg.cond(D[38:, 38:]) > 1e13


def test_error_metrics_definitions():
    f = np.array([1.0, 2.0, 3.0, 4.0]) + 0j
    g = np.array([1.0, 2.5, 3.0, 2.0]) + 0j
    e = T.error_metrics(f, g)
    assert e["max"] == 2.0 and e["mean"] == 0.625 and e["median"] == 0.25
    assert abs(e["rms"] - np.sqrt((0.25 + 4.0) / 4)) < 1e-15
    assert abs(e["rel_rms"] - np.sqrt(4.25 / 30.0)) < 1e-15
    assert e["rel_max"] == 0.5


def test_inputs_generator():
    L, s = 9, 2
    x = inputs.coeffs(L, s, 2, seed=4)
    assert x.shape == (2, L * L)
    assert np.all(x[:, : s * s] == 0) and np.all(x[:, s * s:] != 0)
    assert not np.array_equal(x[0], x[1])
    assert np.array_equal(inputs.coeffs(L, s, 1, seed=5)[0], x[1])
    r = inputs.coeffs(L, 0, 1, seed=1, spectrum="paper", real=True)[0]
    f = T.inverse(r, L, 0)
    assert np.abs(f.imag).max() < 1e-13
    Ls, ss = inputs.uneven_batch(256)
    assert set(Ls) == {128, 256, 512, 1024} and set(ss) == {0, 1, -1, 2, -2}
