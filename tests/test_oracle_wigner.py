"""Pins of the oracle's Wigner d / Delta computation (Sec. 2.2 of the paper).

Each test compares the oracle's Risbo recursion with something outside it: closed forms,
Wigner's explicit sum in exact arithmetic, eqn wignerd_b through Jacobi polynomials,
orthogonality, the symmetry relations, the group law, eqn wigner_sum_reln and the paper's
count of precomputed terms.
"""
import os
from math import sqrt  # noqa: F401  (used by the golden expressions)

import numpy as np
import pytest

from oracle import brute
from oracle import transforms as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def full_index(l, m):
    return l + m


def test_closed_forms_l0_to_l2():
    table = T.delta_quadrant(3)
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "delta_closed_forms.txt")) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 1 + 4 + 9
    for l, mp, m, expr in rows:
        l, mp, m = int(l), int(mp), int(m)
        want = eval(expr, {"sqrt": sqrt})
        got = T.delta_slab(table, l)[mp, m]
        assert abs(got - want) < 1e-15, (l, mp, m, got, want)


@pytest.mark.parametrize("tj", list(range(0, 33)))
def test_risbo_equals_exact_wigner_sum_at_half_pi(tj):
    """Integer and half-integer j up to 16: every entry against the exact explicit sum."""
    D = T.wigner_full(tj)
    E = np.array([[brute.wigner_d_half_pi_exact(tj, 2 * a - tj, 2 * b - tj) for b in range(tj + 1)]
                  for a in range(tj + 1)])
    assert np.abs(D - E).max() < 2e-15 * max(1, tj)


@pytest.mark.parametrize("beta", [0.3, 1.1, 2.0, 2.9])
def test_risbo_at_general_beta_equals_explicit_sum(beta):
    for tj in range(0, 13):
        D = T.wigner_full(tj, beta)
        E = np.array([[brute.wigner_d_sum(tj, 2 * a - tj, 2 * b - tj, beta) for b in range(tj + 1)]
                      for a in range(tj + 1)])
        assert np.abs(D - E).max() < 1e-13


@pytest.mark.parametrize("l", [3, 10, 25, 40])
def test_risbo_equals_jacobi_form(l):
    """Eqn wignerd_b (Jacobi polynomials) against the recursion, at pi/2 and at another beta."""
    for beta in (np.pi / 2, 0.8):
        D = T.wigner_full(2 * l, beta)
        for m in range(-l, l + 1, max(1, l // 7)):
            for n in range(-l, l + 1):
                want = float(brute.wigner_d_jacobi(l, m, n, beta))
                assert abs(D[full_index(l, m), full_index(l, n)] - want) < 1e-12, (l, m, n, beta)


def test_exact_sum_matches_jacobi_form():
    """The two brute-force definitions agree with each other (pins the pins)."""
    for l in range(0, 9):
        for m in range(-l, l + 1):
            for n in range(-l, l + 1):
                a = brute.wigner_d_half_pi_exact(2 * l, 2 * m, 2 * n)
                b = float(brute.wigner_d_jacobi(l, m, n, np.pi / 2))
                assert abs(a - b) < 1e-14


@pytest.mark.parametrize("l", [1, 7, 64, 255])
def test_orthogonality_and_group_law(l):
    """Delta Delta^T = I (unitarity of the real d matrix) and Delta Delta = d(pi),
    with d^l_{mn}(pi) = (-1)^{l-n} delta_{m,-n}."""
    D = T.wigner_full(2 * l)
    n = 2 * l + 1
    assert np.abs(D @ D.T - np.eye(n)).max() < 1e-13 * max(1, np.sqrt(l))
    dpi = np.zeros((n, n))
    for m in range(-l, l + 1):
        dpi[full_index(l, m), full_index(l, -m)] = (-1.0) ** ((l + m) % 2)
    assert np.abs(D @ D - dpi).max() < 1e-13 * max(1, np.sqrt(l))


@pytest.mark.parametrize("l", [2, 5, 30, 200])
def test_symmetry_relations(l):
    """Eqn wignerd_sym1, eqn wignerd_sym6 and its corollary Delta_{m0} = 0 for odd l + m."""
    D = T.wigner_full(2 * l)
    tol = 1e-14 * max(1, l)
    for m in range(-l, l + 1):
        for n in range(-l, l + 1):
            d = D[full_index(l, m), full_index(l, n)]
            assert abs(d - (-1.0) ** ((m - n) % 2) * D[full_index(l, -m), full_index(l, -n)]) < tol
            # eqn wignerd_sym6: d_{-m, n}(pi/2) = (-1)^{l+m} d_{-m,-n}(pi/2)
            assert abs(D[full_index(l, -m), full_index(l, n)]
                       - (-1.0) ** ((l + m) % 2) * D[full_index(l, -m), full_index(l, -n)]) < tol
        if (l + m) % 2 == 1:
            assert abs(D[full_index(l, m), full_index(l, 0)]) < tol


@pytest.mark.parametrize("l", [1, 6, 24])
def test_wigner_sum_relation(l):
    """Eqn wigner_sum_reln: d^l_{mn}(beta) = i^{n-m} sum_{m'} Delta_{m'm} Delta_{m'n} e^{i m' beta}."""
    D = T.wigner_full(2 * l)
    mp = np.arange(-l, l + 1)
    for beta in (0.4, 1.7, 2.6):
        for m in range(-l, l + 1, max(1, l // 5)):
            for n in range(-l, l + 1, max(1, l // 4)):
                s = np.sum(D[:, full_index(l, m)] * D[:, full_index(l, n)] * np.exp(1j * mp * beta))
                val = (1j ** ((n - m) % 4)) * s
                want = float(brute.wigner_d_jacobi(l, m, n, beta))
                assert abs(val.imag) < 1e-13 and abs(val.real - want) < 1e-13


def test_quadrant_table_count_formula():
    """Sec. 4.1: sum_{l=0}^{Lp} (l+1)^2 = Lp^3/3 + 3 Lp^2/2 + 13 Lp/6 + 1 terms."""
    for L in (1, 2, 5, 64, 1024, 2048):
        Lp = L - 1
        paper = Lp ** 3 / 3 + 3 * Lp ** 2 / 2 + 13 * Lp / 6 + 1
        assert int(T.delta_offsets(L)[L]) == round(paper)
    assert T.delta_quadrant(20).size == int(T.delta_offsets(20)[20])


def test_quadrant_table_matches_full_matrices():
    L = 40
    table = T.delta_quadrant(L)
    for l in (0, 1, 17, 39):
        D = T.wigner_full(2 * l)
        q = T.delta_slab(table, l)
        assert np.array_equal(q, D[l:, l:])


def test_large_degree_stays_orthogonal():
    """At l = 1023 (the top degree of the L = 1024 workload) the recursion is still orthogonal."""
    l = 1023
    D = T.wigner_full(2 * l)
    err = np.abs(D @ D.T - np.eye(2 * l + 1)).max()
    assert err < 1e-12
