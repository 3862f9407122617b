"""The paper's triangular forward (eqn matrix_fwd by back substitution) on the GPU against the
oracle's: both exact at small band-limit; at larger L the solve loses accuracy (the paper's
instability) while the quadrature forward stays at machine precision."""
import numpy as np
import pytest
import torch

from oracle import transforms as T
from paper_0807_4494_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def S():
    from paper_0807_4494_gb300 import ssht
    return ssht


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("L,s,B", [(1, 0, 1), (2, 1, 1), (5, 0, 3), (16, 2, 2), (24, -1, 1), (24, 3, 3)])
def test_triangular_forward_exact_at_small_L(L, s, B):
    # the solve amplifies rounding by a factor that grows quickly with L: ~1e7 already at L = 24
    tol = 1e-10 if L <= 16 else 1e-7
    flm = inputs.coeffs(L, s, B, seed=L + 7)
    plan = S().Plan(L, s, B, precision="fp64")
    f = plan.inverse(torch.from_numpy(flm).cuda())
    got = plan.forward_triangular(f).cpu().numpy()
    plan.check()
    fo = f.cpu().numpy()
    for b in range(B):
        assert rel(got[b], flm[b]) < tol
        assert rel(got[b], T.forward_triangular(fo[b], L, s)) < tol


def test_triangular_forward_loses_accuracy_with_L_unlike_the_quadrature():
    errs_tri, errs_quad = {}, {}
    for L in (16, 64, 160):
        flm = inputs.coeffs(L, 2, 1, seed=1, spectrum="paper")
        plan = S().Plan(L, 2, 1, precision="fp64")
        f = plan.inverse(torch.from_numpy(flm).cuda())
        errs_tri[L] = rel(plan.forward_triangular(f).cpu().numpy()[0], flm[0])
        errs_quad[L] = rel(plan.forward(f).cpu().numpy()[0], flm[0])
        plan.check()
    assert errs_tri[16] < 1e-10
    assert errs_tri[160] > 1e4 * errs_tri[16]
    assert max(errs_quad.values()) < 1e-12
    # the oracle's own triangular solve shows the same growth at the largest L
    flm = inputs.coeffs(160, 2, 1, seed=1, spectrum="paper")
    f_or = T.inverse(flm[0], 160, 2)
    assert rel(T.forward_triangular(f_or, 160, 2), flm[0]) > 1e4 * errs_tri[16]


def test_triangular_forward_rejects_non_fp64_plans():
    ssht = S()
    plan = ssht.Plan(8, 0, 1, precision="fp32")
    f = torch.zeros(plan.grid_shape(), dtype=torch.complex64, device="cuda")
    with pytest.raises(ssht.SshtError):
        plan.forward_triangular(f)
