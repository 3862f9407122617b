"""Failure detection without a GPU fault: device-side waits that run out of time and device
allocations that fail, both made to happen on purpose through the library's test hooks.

- A wait gives up after the plan's spin limit (ssht_plan_set_wait_limit); with a limit of 1 ns the
  Risbo recursion's hand-offs and the tensor-core pipeline's waits give up at once.  The kernel
  latches SSHT_ETIMEOUT in the plan, its other CTAs leave at their next wait, copies and MMAs
  already issued are waited for, and the context stays usable: ssht_plan_check reports the timeout,
  and with the default limit restored the next call gives the oracle's result (a cached Delta is
  rebuilt).
- ssht_debug_fail_allocation(n) makes the n-th device allocation fail as an exhausted device
  would; every plan creation it hits returns SSHT_ENOMEM and gives back what it had allocated."""
import numpy as np
import pytest
import torch

from oracle import transforms as T
from paper_0807_4494_gb300 import inputs

pytestmark = pytest.mark.gpu

ETIMEOUT, ENOMEM = -4, -2


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def S():
    from paper_0807_4494_gb300 import ssht
    return ssht


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def test_recursion_hand_off_timeout_is_latched_and_the_plan_recovers():
    ssht = S()
    L = 300
    plan = ssht.Plan(L, 0, 1, recursion="risbo")
    plan.set_wait_limit(1)
    plan.wigner_delta()
    with pytest.raises(ssht.SshtError) as e:
        plan.check()
    assert e.value.code == ETIMEOUT
    plan.check()  # the status was cleared by the check that reported it
    plan.set_wait_limit(0)
    tab = plan.wigner_delta().cpu().numpy()
    plan.check()
    assert np.abs(tab - T.delta_quadrant(L)).max() < 1e-13


@pytest.mark.parametrize("delta_mode", ["recompute", "cache"])
def test_contraction_pipeline_timeout_is_latched_and_the_plan_recovers(delta_mode):
    ssht = S()
    L, s, B = 96, 2, 8
    flm = inputs.coeffs(L, s, B, seed=4)
    x = torch.from_numpy(flm).to(torch.complex64).cuda()
    plan = ssht.Plan(L, s, B, precision="tf32x3", delta_mode=delta_mode)
    plan.set_wait_limit(1)
    plan.inverse(x)
    with pytest.raises(ssht.SshtError) as e:
        plan.check()
    assert e.value.code == ETIMEOUT
    plan.set_wait_limit(0)
    f = plan.inverse(x)
    back = plan.forward(f)
    plan.check()
    f = f.cpu().numpy()
    for b in (0, B - 1):
        assert rel(f[b], T.inverse(flm[b], L, s)) < 1e-6
        assert rel(back[b].cpu().numpy(), T.forward(f[b].astype(np.complex128), L, s)) < 1e-6


def _free_bytes():
    import gc
    gc.collect()  # plans of earlier tests give their memory back when collected
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("precision", ["tf32x3", "fp64"])
def test_allocation_failures_during_plan_creation_release_everything(precision):
    ssht = S()
    L, s, B = 40, 1, 3
    base = _free_bytes()
    created = False
    try:
        for n in range(1, 64):
            ssht.ssht_debug_fail_allocation(n)
            try:
                plan = ssht.Plan(L, s, B, precision=precision)
            except ssht.SshtError as e:
                assert e.code == ENOMEM, (n, e)
                assert _free_bytes() > base - (8 << 20), n  # nothing of the failed plan is kept
                continue
            created = True  # n is past the plan's last allocation: the hook did not fire
            ssht.ssht_debug_fail_allocation(0)
            plan.close()
            break
    finally:
        ssht.ssht_debug_fail_allocation(0)
    assert created and n > 5
    assert _free_bytes() > base - (8 << 20)
    # the library still works
    flm = inputs.coeffs(L, s, B, seed=2)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    plan = ssht.Plan(L, s, B, precision=precision)
    f = plan.inverse(torch.from_numpy(flm).to(dt).cuda()).cpu().numpy()
    plan.check()
    plan.close()
    assert rel(f, T.inverse(flm, L, s)) < (1e-12 if precision == "fp64" else 1e-6)


def test_allocation_failure_during_group_creation():
    ssht = S()
    base = _free_bytes()
    try:
        ssht.ssht_debug_fail_allocation(7)
        with pytest.raises(ssht.SshtError) as e:
            ssht.Group([16, 32, 32], [0, 1, -1], precision="fp32", tune=False)
        assert e.value.code == ENOMEM
    finally:
        ssht.ssht_debug_fail_allocation(0)
    assert _free_bytes() > base - (8 << 20)
