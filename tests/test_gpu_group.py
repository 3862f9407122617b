"""Groups of fields with uneven band-limit and spin (the uneven-batch configuration, scaled
down): parity of every field with the FP64 oracle, one CUDA graph for the whole group, shared
Delta tables (cache = recompute), tuned buckets."""
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


def make_case(n=24, Lset=(16, 32, 48, 64), seed=0):
    rng = np.random.default_rng(seed)
    Ls = [int(x) for x in rng.choice(Lset, n)]
    ss = [int(x) for x in rng.choice((0, 1, -1, 2, -2), n)]
    flms = [inputs.coeffs(L, s, 1, seed=seed * 1000 + i)[0] for i, (L, s) in enumerate(zip(Ls, ss))]
    return Ls, ss, flms


@pytest.mark.parametrize("precision,tune,tol", [("fp32", True, 2e-6), ("tf32x3", False, 1e-6), ("fp64", False, 1e-12)])
def test_group_matches_oracle_per_field(precision, tune, tol):
    Ls, ss, flms = make_case()
    g = S().Group(Ls, ss, precision=precision, tune=tune)
    dt = g.dtype
    flat = g.pack_coeffs([torch.from_numpy(x).to(dt).cuda() for x in flms])
    f = g.inverse(flat)
    back = g.forward(f)
    adj = g.adjoint(f)
    g.check()
    fs, bs, As = g.unpack_grid(f), g.unpack_coeffs(back), g.unpack_coeffs(adj)
    assert sum(b[2] for b in g.buckets()) == len(Ls)
    for i, (L, s) in enumerate(zip(Ls, ss)):
        fi = fs[i].cpu().numpy()
        assert rel(fi, T.inverse(flms[i], L, s)) < tol
        assert rel(bs[i].cpu().numpy(), T.forward(fi.astype(np.complex128), L, s)) < tol
        assert rel(As[i].cpu().numpy(), T.adjoint(fi.astype(np.complex128), L, s)) < tol


def config4_case(per_bucket=2, seed=0):
    """The uneven-batch configuration at its own band-limits, scaled down in count: every (L, s)
    bucket with L in {128, 256, 512, 1024} and s in {0, +-1, +-2} holds `per_bucket` fields,
    Re/Im iid N(0,1), in a shuffled caller order."""
    rng = np.random.default_rng(seed)
    pairs = [(L, s) for L in (128, 256, 512, 1024) for s in (0, 1, -1, 2, -2)] * per_bucket
    order = rng.permutation(len(pairs))
    Ls = [pairs[i][0] for i in order]
    ss = [pairs[i][1] for i in order]
    flms = [inputs.coeffs(L, s, 1, seed=seed * 1000 + i)[0] for i, (L, s) in enumerate(zip(Ls, ss))]
    return Ls, ss, flms


@pytest.mark.slow
@pytest.mark.parametrize("precision,tune", [("fp32", True), ("tf32x3", False)])
def test_group_at_uneven_batch_band_limits(precision, tune):
    """Shared Delta per L, per-bucket streams, the tuner's choice and the graph replay at the
    uneven batch's own band-limits: every field of the L <= 256 buckets and the first field of
    every L = 512 and L = 1024 bucket, inverse (from the graph), forward and adjoint."""
    Ls, ss, flms = config4_case()
    g = S().Group(Ls, ss, precision=precision, tune=tune)
    dt = g.dtype
    flat = g.pack_coeffs([torch.from_numpy(x).to(dt).cuda() for x in flms])
    f_s, b_s = g.empty_grid(), g.empty_coeffs()
    g.capture(flat, f_s, b_s)
    g.replay()
    adj = g.adjoint(f_s)
    g.check()
    fs, bs, As = g.unpack_grid(f_s), g.unpack_coeffs(b_s), g.unpack_coeffs(adj)
    seen = set()
    for i, (L, s) in enumerate(zip(Ls, ss)):
        if L > 256 and (L, s) in seen:
            continue
        seen.add((L, s))
        fi = fs[i].cpu().numpy()
        assert rel(fi, T.inverse(flms[i], L, s)) < 2e-6, ("inverse", L, s)
        g64 = fi.astype(np.complex128)
        assert rel(bs[i].cpu().numpy(), T.forward(g64, L, s)) < 2e-6, ("forward", L, s)
        assert rel(As[i].cpu().numpy(), T.adjoint(g64, L, s)) < 2e-6, ("adjoint", L, s)
    assert len(seen) == 20


def test_group_graph_replay_and_cache_mode():
    Ls, ss, flms = make_case(n=16, seed=1)
    g = S().Group(Ls, ss, precision="fp32", tune=True)
    flat = g.pack_coeffs([torch.from_numpy(x).to(torch.complex64).cuda() for x in flms])
    f_e = g.inverse(flat)
    b_e = g.forward(f_e)
    f_s, b_s = g.empty_grid(), g.empty_coeffs()
    g.capture(flat, f_s, b_s)
    for _ in range(2):
        f_s.zero_()
        b_s.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(f_s, f_e)
        assert torch.equal(b_s, b_e)
    g.check()
    # the same buckets with the tables made at creation give the same numbers
    gc = S().Group(Ls, ss, precision="fp32", delta_mode="cache", tune=False)
    fc = gc.inverse(flat)
    gplain = S().Group(Ls, ss, precision="fp32", tune=False)
    assert torch.equal(fc, gplain.inverse(flat))
    gc.check()


def test_group_layout_and_errors():
    ssht = S()
    Ls, ss = [8, 4, 8, 4, 6], [0, 1, 0, -1, 2]
    g = ssht.Group(Ls, ss, precision="fp64", tune=False)
    # group order: by L then s, stable in the caller's index
    assert g.order == [1, 3, 4, 0, 2] or [Ls[i] for i in g.order] == sorted(Ls)
    assert g.coff[-1] == sum(L * L for L in Ls)
    assert g.goff[-1] == sum(L * (2 * L - 1) for L in Ls)
    with pytest.raises(ssht.SshtError):
        ssht.Group([4, 4], [0, 4])        # |s| >= L
    big = ssht.Group([4] * 70, [0] * 70, precision="tf32x3", tune=False)  # > 64 fields: two GEMM slices
    assert big.bucket_tile_config(0)["slice"] == 64
