"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Error measure: max-norm relative error max|x - x_oracle| / max|x_oracle|.  FP64 bound: 1e-12
(the benchmark spec's bound for the FP64 path is 1e-11 at L <= 512).  FP32 plans: 2e-6.
"""
import numpy as np
import pytest
import torch

from oracle import transforms as T
from paper_0807_4494_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def S():
    from paper_0807_4494_gb300 import ssht
    return ssht


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def dev(x, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


def random_grid(L, B, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, L, 2 * L - 1)) + 1j * rng.standard_normal((B, L, 2 * L - 1))


RECURSIONS = ["column", "risbo"]


@pytest.mark.parametrize("recursion", RECURSIONS)
@pytest.mark.parametrize("L", [1, 2, 3, 8, 32, 33, 64, 65, 100, 257])
def test_delta_table_matches_oracle(L, recursion):
    plan = S().Plan(L, 0, 1, recursion=recursion)
    got = plan.wigner_delta().cpu().numpy()
    plan.check()
    want = T.delta_quadrant(L)
    assert got.shape == want.shape
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("recursion", RECURSIONS)
def test_delta_table_top_degrees_at_L1024(recursion):
    L = 1024
    plan = S().Plan(L, 0, 1, recursion=recursion)
    tab = plan.wigner_delta().cpu().numpy()
    plan.check()
    for l in (1023, 640):
        full = T.wigner_full(2 * l)
        assert np.abs(T.delta_slab(tab, l) - full[l:, l:]).max() < 5e-13


def test_delta_table_degrees_of_L2048():
    """Band-limit 2048 (the column method's scaled variant: first-row entries of high degrees are
    below the FP64 normal range and start with a per-lane exponent): whole degrees against the
    oracle's full-matrix Risbo recursion, copied off the 22.9 GB device table one degree at a time."""
    L = 2048
    plan = S().Plan(L, 0, 1)
    tab = plan.wigner_delta()
    plan.check()
    off = T.delta_offsets(L)
    for l in (1100, 2047):
        got = tab[int(off[l]):int(off[l + 1])].cpu().numpy().reshape(l + 1, l + 1)
        full = T.wigner_full(2 * l)
        assert np.abs(got - full[l:, l:]).max() < 5e-13


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("tf32x3", 1e-6)])
def test_transforms_with_the_risbo_recursion(precision, tol):
    """Plans with SSHT_FLAG_RISBO (the paper's recursion) give the oracle's transforms too, and
    agree with the default plans to rounding."""
    L, s, B = 97, 2, 3
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    flm = inputs.coeffs(L, s, B, seed=17)
    a = S().Plan(L, s, B, precision=precision, recursion="risbo")
    b = S().Plan(L, s, B, precision=precision)
    fa = a.inverse(dev(flm, dt))
    ba = a.forward(fa).cpu().numpy()
    fb = b.inverse(dev(flm, dt)).cpu().numpy()
    a.check()
    b.check()
    fa = fa.cpu().numpy()
    for k in range(B):
        f_or = T.inverse(flm[k], L, s)
        assert rel(fa[k], f_or) < tol
        assert rel(ba[k], T.forward(fa[k].astype(np.complex128), L, s)) < tol
    assert rel(fa, fb) < tol


@pytest.mark.parametrize("L,s,B", [(1, 0, 1), (2, 0, 1), (2, 1, 2), (5, 0, 3), (8, 2, 1), (8, -2, 2), (17, 3, 1),
                                   (33, -1, 3), (40, 39, 1), (64, 0, 2), (97, 5, 1)])
def test_inverse_fp64(L, s, B):
    flm = inputs.coeffs(L, s, B, seed=L + s)
    plan = S().Plan(L, s, B)
    f = plan.inverse(dev(flm)).cpu().numpy()
    plan.check()
    assert rel(f, T.inverse(flm, L, s)) < TOL64


@pytest.mark.parametrize("L,s,B", [(1, 0, 1), (2, 1, 1), (5, 0, 3), (8, 2, 2), (17, -3, 1), (33, 1, 3), (40, 39, 1),
                                   (64, 2, 1), (97, -5, 2)])
def test_forward_fp64_band_limited(L, s, B):
    flm = inputs.coeffs(L, s, B, seed=3 * L + s)
    f = T.inverse(flm, L, s)
    plan = S().Plan(L, s, B)
    got = plan.forward(dev(f)).cpu().numpy()
    plan.check()
    assert rel(got, T.forward(f, L, s)) < TOL64
    assert rel(got, flm) < TOL64


@pytest.mark.parametrize("L,s,B", [(2, 0, 1), (9, 1, 2), (30, -2, 1), (64, 3, 2)])
def test_forward_fp64_arbitrary_samples(L, s, B):
    """Samples that are not band-limited: both sides apply the same linear map (including the
    zeroed theta = pi sample of odd columns)."""
    g = random_grid(L, B, seed=L)
    plan = S().Plan(L, s, B)
    got = plan.forward(dev(g)).cpu().numpy()
    plan.check()
    assert rel(got, T.forward(g, L, s)) < TOL64


@pytest.mark.parametrize("L,s,B", [(1, 0, 1), (4, 0, 1), (9, 2, 2), (31, -1, 1), (64, 2, 3)])
def test_adjoint_fp64(L, s, B):
    g = random_grid(L, B, seed=7 * L)
    plan = S().Plan(L, s, B)
    got = plan.adjoint(dev(g)).cpu().numpy()
    plan.check()
    assert rel(got, T.adjoint(g, L, s)) < TOL64


def test_config1_L64_s2_roundtrip():
    """L = 64, s = 2, Re/Im iid N(0,1), seed 0: inverse to the grid, then forward."""
    L, s = 64, 2
    flm = inputs.coeffs(L, s, 1, seed=0)
    plan = S().Plan(L, s, 1)
    f = plan.inverse(dev(flm))
    back = plan.forward(f).cpu().numpy()
    plan.check()
    assert rel(f.cpu().numpy(), T.inverse(flm, L, s)) < TOL64
    assert rel(back, flm) < TOL64


@pytest.mark.parametrize("s", [0, 2])
def test_config2_L512(s):
    L = 512
    flm = inputs.coeffs(L, s, 1, seed=0)
    plan = S().Plan(L, s, 1)
    f = plan.inverse(dev(flm))
    back = plan.forward(f).cpu().numpy()
    plan.check()
    f_or = T.inverse(flm, L, s)
    assert rel(f.cpu().numpy(), f_or) < 1e-11
    assert rel(back, T.forward(f_or, L, s)) < 1e-11
    assert rel(back, flm) < 1e-11


@pytest.mark.parametrize("L,s,B", [(16, 0, 1), (64, 2, 3), (128, -1, 2)])
def test_fp32_plan(L, s, B):
    flm = inputs.coeffs(L, s, B, seed=11)
    plan = S().Plan(L, s, B, precision="fp32")
    f = plan.inverse(dev(flm, torch.complex64))
    back = plan.forward(f).cpu().numpy()
    adj = plan.adjoint(f).cpu().numpy()
    plan.check()
    f_or = T.inverse(flm, L, s)
    assert rel(f.cpu().numpy(), f_or) < TOL32
    assert rel(back, flm) < TOL32
    assert rel(adj, T.adjoint(f_or, L, s)) < TOL32


def test_many_rows_fp32():
    """batch * (2L-1) > 65535 rows (the row-wise kernels must not rely on gridDim.y)."""
    L, s, B = 256, 1, 129
    flm = inputs.coeffs(L, s, B, seed=0)
    plan = S().Plan(L, s, B, precision="fp32")
    f = plan.inverse(dev(flm, torch.complex64))
    back = plan.forward(f).cpu().numpy()
    adj = plan.adjoint(f).cpu().numpy()
    plan.check()
    f = f.cpu().numpy()
    for b in (0, B - 1):
        f_or = T.inverse(flm[b], L, s)
        assert rel(f[b], f_or) < TOL32
        assert rel(back[b], flm[b]) < TOL32
        assert rel(adj[b], T.adjoint(f_or, L, s)) < TOL32


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_headline_band_limit_two_fields(prec):
    """L = 1024 (torus length 2047, shared-memory Bluestein with M = 4096), s = 2, CMB-like spectrum."""
    L, s, B = 1024, 2, 2
    flm = inputs.coeffs(L, s, B, seed=3, spectrum="cmb")
    plan = S().Plan(L, s, B, precision=prec)
    f = plan.inverse(dev(flm, torch.complex64))
    back = plan.forward(f).cpu().numpy()
    plan.check()
    f = f.cpu().numpy()
    f_or = T.inverse(flm[1], L, s)
    assert rel(f[1], f_or) < 1e-6
    assert rel(back[1], T.forward(f[1].astype(np.complex128), L, s)) < 1e-6


def test_host_pointers_match_device_pointers():
    L, s, B = 24, 1, 2
    flm = inputs.coeffs(L, s, B, seed=5)
    plan = S().Plan(L, s, B)
    f_dev = plan.inverse(dev(flm))
    f_host = plan.inverse(torch.from_numpy(flm))
    assert not f_host.is_cuda
    assert torch.equal(f_dev.cpu(), f_host)
    back_host = plan.forward(f_host)
    assert torch.equal(back_host, plan.forward(f_dev).cpu())
    plan.check()


@pytest.mark.parametrize("precision,real", [("tf32x3", False), ("fp32", False), ("fp64", False), ("tf32x3", True)])
def test_page_locked_host_inputs_match_device_inputs(precision, real):
    """Page-locked host inputs are copied to plan-owned device memory by the copy engines before the
    call's kernels read them: the results equal those of device inputs bit for bit (tensor-core,
    FP32 and FP64 plans, real-field packing; inverse, forward and adjoint)."""
    L, s, B = 40, 0 if real else 2, 3
    plan = S().Plan(L, s, B, precision=precision, real=real)
    flm = inputs.coeffs(L, s, B, seed=8, spectrum="paper", real=True) if real else inputs.coeffs(L, s, B, seed=8)
    x = torch.from_numpy(flm).to(plan.dtype)
    f_dev = plan.inverse(x.cuda())
    f_pin = plan.inverse(x.pin_memory()).cuda()
    torch.cuda.synchronize()
    assert torch.equal(f_dev, f_pin)
    g_pin = f_dev.cpu().pin_memory()
    assert torch.equal(plan.forward(g_pin).cuda(), plan.forward(f_dev))
    assert torch.equal(plan.adjoint(g_pin).cuda(), plan.adjoint(f_dev))
    plan.check()


def test_host_input_call_runs_on_the_current_stream():
    """With a side stream current, a call whose input is page-locked host memory runs on that
    stream like the calls with device data, so that an inverse from host memory followed by a
    forward of its device result (the serving pattern, one plan per stream) sees the inverse
    finished: results equal those of the default stream bit for bit."""
    L, s, B = 64, 2, 4
    plan = S().Plan(L, s, B, precision="tf32x3")
    x = torch.from_numpy(inputs.coeffs(L, s, B, seed=4)).to(plan.dtype)
    f_ref = plan.inverse(x.cuda())
    b_ref = plan.forward(f_ref)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    h_in = x.pin_memory()
    h_out = torch.empty(plan.coeff_shape(), dtype=plan.dtype).pin_memory()
    grid = torch.empty_like(f_ref)
    with torch.cuda.stream(side):
        for _ in range(3):
            plan.inverse(h_in, out=grid)
            plan.forward(grid, out=h_out)
    torch.cuda.synchronize()
    assert torch.equal(grid, f_ref)
    assert torch.equal(h_out.cuda(), b_ref)
    plan.check()


def test_cache_mode_equals_recompute_mode():
    L, s, B = 48, -2, 2
    flm = dev(inputs.coeffs(L, s, B, seed=9))
    a = S().Plan(L, s, B, delta_mode="recompute")
    b = S().Plan(L, s, B, delta_mode="cache")
    fa, fb = a.inverse(flm), b.inverse(flm)
    assert torch.equal(fa, fb)
    assert torch.equal(a.forward(fa), b.forward(fb))
    a.check()
    b.check()


def test_adjoint_dot_product_on_gpu():
    L, s = 80, 2
    plan = S().Plan(L, s, 1)
    a = dev(inputs.coeffs(L, s, 1, seed=2))
    g = dev(random_grid(L, 1, seed=3))
    lhs = torch.vdot(plan.inverse(a).flatten(), g.flatten())
    rhs = torch.vdot(a.flatten(), plan.adjoint(g).flatten())
    assert abs(complex(lhs - rhs)) < 1e-12 * abs(complex(lhs))


def test_autograd_backward_is_adjoint_and_matches_finite_differences():
    """Gradient of a real loss through the differentiable inverse at L = 128 (random direction,
    seed 1, central differences with h = 1e-3 and 1e-4)."""
    ssht = S()
    L, s = 128, 2
    plan = ssht.Plan(L, s, 1)
    a = dev(inputs.coeffs(L, s, 1, seed=0)).requires_grad_(True)
    w = dev(random_grid(L, 1, seed=4))

    def loss(x):
        f = ssht.inverse(x, plan)
        return (f * w.conj()).real.sum() + 0.5 * (f.abs() ** 2).sum()

    val = loss(a)
    val.backward()
    grad = a.grad.detach()
    rng = np.random.default_rng(1)
    d = dev(rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape))
    d[:, : s * s] = 0
    with torch.no_grad():
        for h in (1e-3, 1e-4):
            fd = (loss(a + h * d) - loss(a - h * d)) / (2 * h)
            # torch's gradient of a real loss is dl/dRe + i dl/dIm, so dl = Re <grad, d>
            an = torch.vdot(grad.flatten(), d.flatten()).real
            assert abs(float(fd) - float(an)) < 1e-6 * max(1.0, abs(float(an)))
    plan.check()


@pytest.mark.slow
def test_full_size_single_field_L1024_fp64():
    """The headline band-limit L = 1024, s = 2, CMB-like spectrum, one field in FP64."""
    L, s = 1024, 2
    flm = inputs.coeffs(L, s, 1, seed=0, spectrum="cmb")
    plan = S().Plan(L, s, 1)
    f = plan.inverse(dev(flm)).cpu().numpy()
    f_or = T.inverse(flm, L, s)
    assert rel(f, f_or) < 1e-11
    back = plan.forward(dev(f_or)).cpu().numpy()
    plan.check()
    assert rel(back, T.forward(f_or, L, s)) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3"])
def test_calls_capture_into_a_cuda_graph(precision):
    """inverse + forward (recursion forked onto the plan's second stream and joined) capture into
    one CUDA graph whose replays reproduce the eager results bit for bit."""
    L, s, B = 48, 2, 3
    plan = S().Plan(L, s, B, precision=precision)
    dt = plan.dtype
    flm = torch.from_numpy(inputs.coeffs(L, s, B, seed=9)).to(dt).cuda()
    f_eager = plan.inverse(flm)
    b_eager = plan.forward(f_eager)
    f_static = torch.empty_like(f_eager)
    b_static = torch.empty_like(b_eager)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.inverse(flm, out=f_static)
        plan.forward(f_static, out=b_static)
    for _ in range(2):
        f_static.zero_()
        b_static.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(f_static, f_eager)
        assert torch.equal(b_static, b_eager)
    plan.check()


@pytest.mark.parametrize("precision", ["fp64", "tf32x3", "bf16x6"])
def test_plans_of_different_sizes_interleave(precision):
    """Kernel launch limits are process-wide: a plan made after a larger one must not stop the
    larger one from launching (shared-memory sizes differ with L and the batch)."""
    big = S().Plan(200, 1, 40, precision=precision)
    dt = big.dtype
    flm_big = torch.from_numpy(inputs.coeffs(200, 1, 40, seed=3)).to(dt).cuda()
    f1 = big.inverse(flm_big)
    small = S().Plan(16, 0, 1, precision=precision)
    small.inverse(torch.from_numpy(inputs.coeffs(16, 0, 1, seed=4)).to(dt).cuda())
    f2 = big.inverse(flm_big)
    assert torch.equal(f1, f2)
    big.check()
    small.check()


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_back_to_back_calls_without_host_sync(precision):
    """A call's recursion may start while the previous call's torus stage still runs; calls queued
    back to back (with a Delta table copy between them) give what synchronised calls give."""
    L, s, B = 96, 1, 4
    plan = S().Plan(L, s, B, precision=precision)
    dt = plan.dtype
    flm = torch.from_numpy(inputs.coeffs(L, s, B, seed=21)).to(dt).cuda()
    f_ref = plan.inverse(flm)
    torch.cuda.synchronize()
    b_ref = plan.forward(f_ref)
    torch.cuda.synchronize()
    t_ref = plan.wigner_delta()
    torch.cuda.synchronize()
    outs = []
    for _ in range(3):
        f = plan.inverse(flm)
        t = plan.wigner_delta()
        b = plan.forward(f)
        a = plan.adjoint(f)
        outs.append((f, t, b, a))
    torch.cuda.synchronize()
    plan.check()
    a_ref = plan.adjoint(f_ref)
    torch.cuda.synchronize()
    for f, t, b, a in outs:
        assert torch.equal(f, f_ref)
        assert torch.equal(t, t_ref)
        assert torch.equal(b, b_ref)
        assert torch.equal(a, a_ref)


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x6", "fp32"])
def test_pipelined_calls_match_synchronised_calls(precision):
    """Calls queued back to back let the next call's recursion start before the previous call
    has finished (it waits only for the readers of what it overwrites); the results must equal
    those of calls separated by host synchronisation."""
    L, s, B = 80, 2, 6
    plan = S().Plan(L, s, B, precision=precision)
    flm = torch.from_numpy(inputs.coeffs(L, s, B, seed=31)).to(plan.dtype).cuda()
    f_ref = plan.inverse(flm)
    torch.cuda.synchronize()
    b_ref = plan.forward(f_ref)
    torch.cuda.synchronize()
    a_ref = plan.adjoint(f_ref)
    torch.cuda.synchronize()
    res = []
    for _ in range(4):
        f = plan.inverse(flm)
        res.append((f, plan.forward(f), plan.adjoint(f), plan.forward(f)))
    torch.cuda.synchronize()
    plan.check()
    for f, b, a, b2 in res:
        assert torch.equal(f, f_ref)
        assert torch.equal(b, b_ref)
        assert torch.equal(a, a_ref)
        assert torch.equal(b2, b_ref)


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_profile_totals_and_trace(precision):
    """Stage timing: the trace lists every bracket once, each stream's brackets in order and
    without overlap, the recursion (and, for the tensor-core path, the A packing) on the plan's
    second stream; its per-stage sums equal the totals read afterwards."""
    L, s, B = 96, 2, 4
    plan = S().Plan(L, s, B, precision=precision)
    flm = torch.from_numpy(inputs.coeffs(L, s, B, seed=3)).to(plan.dtype).cuda()
    plan.inverse(flm)
    plan.profile(True)
    for _ in range(2):
        f = plan.inverse(flm)
        plan.forward(f)
    trace = plan.profile_trace()
    assert trace and min(t0 for _, _, t0, _ in trace) == 0.0
    for name, lane, t0, t1 in trace:
        assert name in S().STAGES and lane in (0, 1) and 0.0 <= t0 <= t1
    for lane in (0, 1):
        spans = [(t0, t1) for _, ln, t0, t1 in trace if ln == lane]
        assert all(a[1] <= b[0] + 1e-3 for a, b in zip(spans, spans[1:]))
    aux = {name for name, lane, _, _ in trace if lane == 1}
    if precision == "fp64":
        # one table recursion per call
        assert aux == {"delta"}
        assert sum(1 for name, _, _, _ in trace if name == "delta") == 4
    else:
        # 3xTF32: the recursions write the A tiles of both directions themselves, one per call
        assert aux == {"delta", "delta_inverse"}
        assert sum(1 for name, _, _, _ in trace if name == "delta") == 2
        assert sum(1 for name, _, _, _ in trace if name == "delta_inverse") == 2
    # the trace was folded into the totals
    totals, launches = plan.profile_read()
    assert launches > 0
    for name in S().STAGES:
        spans = [t1 - t0 for n, _, t0, t1 in trace if n == name]
        assert totals[name][1] == len(spans)
        assert totals[name][0] == pytest.approx(sum(spans), rel=1e-3, abs=1e-3)
    assert plan.profile_trace() == []
    plan.check()
