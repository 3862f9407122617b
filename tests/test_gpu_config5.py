"""High band-limit: L = 2048, s = 2, B = 16 fields with the CMB-like spectrum, through the
split-BF16 and 3xTF32 tensor-core paths and the plain FP64 path (the recursion runs in chunks at
this size, the 3xTF32 plan's tile-writing recursions carry a per-lane exponent, and the torus
passes use 8192-point FFTs).  Sampled parity with the FP64 oracle on field 0."""
import numpy as np
import pytest
import torch

from oracle import transforms as T
from paper_0807_4494_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

L, SPIN, B = 2048, 2, 16


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def case():
    flm = inputs.coeffs(L, SPIN, B, seed=0, spectrum="cmb")
    return flm, T.inverse(flm[0], L, SPIN)


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("precision,tol", [("bf16x6", 2e-6), ("tf32x3", 2e-6), ("fp64", 1e-10)])
def test_L2048_inverse_and_roundtrip(case, precision, tol):
    from paper_0807_4494_gb300 import ssht
    flm, f_or = case
    plan = ssht.Plan(L, SPIN, B, precision=precision)
    x = torch.from_numpy(flm).to(plan.dtype).cuda()
    f = plan.inverse(x)
    back = plan.forward(f)
    plan.check()
    f0 = f[0].cpu().numpy()
    assert rel(f0, f_or) < tol
    assert float((back - x).abs().max() / x.abs().max()) < 2 * tol
    if precision != "fp64":
        fw = T.forward(f0.astype(np.complex128), L, SPIN)
        assert rel(back[0].cpu().numpy(), fw) < tol
    del plan, f, back
    torch.cuda.empty_cache()
