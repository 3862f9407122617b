"""Real spin-0 fields (SSHT_FLAG_REAL): two real fields per complex transform.  Parity with the
FP64 oracle, equality with the complex path, odd field counts, and the paper's real workload
(U[-1,1] coefficients with the reality condition)."""
import numpy as np
import pytest
import torch

from oracle import transforms as T
from paper_0807_4494_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6, "tf32x3": 1e-6, "bf16x6": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def S():
    from paper_0807_4494_gb300 import ssht
    return ssht


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3", "bf16x6"])
@pytest.mark.parametrize("L,B,spectrum", [(1, 1, "flat"), (9, 5, "paper"), (64, 2, "flat"), (130, 3, "cmb")])
def test_real_fields_match_oracle(precision, L, B, spectrum):
    tol = TOL[precision]
    flm = inputs.coeffs(L, 0, B, seed=L + B, spectrum=spectrum, real=True)
    plan = S().Plan(L, 0, B, precision=precision, real=True)
    x = torch.from_numpy(flm).to(plan.dtype).cuda()
    f = plan.inverse(x)
    assert f.dtype == plan.grid_dtype and not f.is_complex()
    back = plan.forward(f)
    adj = plan.adjoint(f)
    plan.check()
    fo, bo, ao = f.cpu().numpy(), back.cpu().numpy(), adj.cpu().numpy()
    for b in range(B):
        f_or = T.inverse(flm[b], L, 0)
        assert np.abs(f_or.imag).max() <= 1e-12 * np.abs(f_or).max()
        assert rel(fo[b], f_or.real) < tol
        g = fo[b].astype(np.complex128)
        assert rel(bo[b], T.forward(g, L, 0)) < tol
        assert rel(ao[b], T.adjoint(g, L, 0)) < tol
        assert rel(bo[b], flm[b]) < 2 * tol


def test_real_plan_equals_complex_plan():
    L, B = 48, 4
    flm = inputs.coeffs(L, 0, B, seed=3, real=True)
    x = torch.from_numpy(flm).cuda()
    pr = S().Plan(L, 0, B, precision="fp64", real=True)
    pc = S().Plan(L, 0, B, precision="fp64")
    fr, fc = pr.inverse(x), pc.inverse(x)
    assert float((fr - fc.real).abs().max()) < 1e-13 * float(fc.abs().max())
    br, bc = pr.forward(fr), pc.forward(fc.real.to(torch.complex128).contiguous())
    assert float((br - bc).abs().max()) < 1e-13 * float(bc.abs().max())
    # the triangular forward is only accurate at small band-limits (the paper's instability)
    flm = inputs.coeffs(12, 0, 3, seed=5, real=True)
    x = torch.from_numpy(flm).cuda()
    pr = S().Plan(12, 0, 3, precision="fp64", real=True)
    tr = pr.forward_triangular(pr.inverse(x))
    assert float((tr - x).abs().max()) < 1e-10 * float(x.abs().max())


def test_real_flag_needs_spin_zero():
    ssht = S()
    with pytest.raises(ssht.SshtError):
        ssht.Plan(16, 1, 2, real=True)


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
@pytest.mark.parametrize("L,s,B", [(33, 2, 3), (64, -1, 4), (20, 0, 2)])
def test_spin_pairs_give_both_spins_from_one_transform(precision, L, s, B):
    """SSHT_FLAG_SPIN_PAIR: for each field f of spin s, the forward and the adjoint return the spin-s
    coefficients of f and the spin -s coefficients of conj(f) (the pair f_s* = f_{-s}) from one
    spin-s transform; every field of both halves against the oracle's transform of f (spin s) and
    of conj(f) (spin -s).  The inverse of the pair reads its spin-s half."""
    ssht = S()
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    flm = inputs.coeffs(L, s, B, seed=L + 7)
    f = np.ascontiguousarray(T.inverse(flm, L, s))
    g = np.random.default_rng(3).standard_normal(f.shape) + 1j * np.random.default_rng(4).standard_normal(f.shape)
    plan = ssht.Plan(L, s, B, precision=precision, spin_pair=True)
    fwd = plan.forward(torch.from_numpy(f).to(dt).cuda()).cpu().numpy()
    adj = plan.adjoint(torch.from_numpy(g).to(dt).cuda()).cpu().numpy()
    pair_in = np.stack([flm, np.zeros_like(flm)], axis=1)  # the spin -s half is not read
    inv = plan.inverse(torch.from_numpy(pair_in).to(dt).cuda()).cpu().numpy()
    plan.check()
    assert fwd.shape == (B, 2, L * L)
    tol = TOL[precision]
    for b in range(B):
        assert rel(fwd[b, 0], T.forward(f[b], L, s)) < tol
        assert rel(fwd[b, 1], T.forward(np.conj(f[b]), L, -s)) < tol
        assert rel(adj[b, 0], T.adjoint(g[b], L, s)) < tol
        assert rel(adj[b, 1], T.adjoint(np.conj(g[b]), L, -s)) < tol
        assert rel(inv[b], f[b]) < tol
