"""The bounded device waits, exercised on purpose without a fault.

fmm_plan_debug_timeout makes the next prefix-schedule M2L launch leave the
first activation stage of every CTA unloaded.  Nothing is copied into that
stage and no MMA reads it, so when the issuers' wait on it reaches its 2 s
limit nothing is in flight: each CTA lets its own weight copies land, frees
its tensor memory and exits, the later launches of the solve see the flag and
skip their work.  fmm_check must then report FMM_ERR_TIMEOUT with the
issuers' activation wait, or the epilogue's wait on those issuers'
accumulators, among the sites (both wait on the starved stage; the epilogue
starts waiting first, and a waiter that finds the flag already set leaves
without adding its own site, so which of the two is recorded depends on
when each checks its clock), clear the flag, and the next ordinary solve on
the same plan must match the oracle.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2606_13793_gb300 as fmm  # noqa: E402
from paper_2606_13793_gb300 import _build, inputs  # noqa: E402

W_MMA_A = 2  # wait sites of the issuers' activation wait and of the epilogue (the kernels' WaitSite numbering)
W_EPI = 4


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    assert torch.cuda.is_available()


def test_timeout_is_reported_and_the_plan_recovers(orc):
    n = 128
    rho32 = inputs.lognormal(n, seed=23)
    rho = torch.from_numpy(rho32).cuda()
    plan = fmm.FMMPlan((n, n, n), 6, 4, "bf16x3")
    plan.set_tc_schedule("m2l", "prefix")
    plan.solve(rho)
    plan.check()  # an ordinary solve first: no flag

    plan.debug_timeout()
    t0 = time.perf_counter()
    plan.solve(rho)
    with pytest.raises(fmm.FMMError) as e:
        plan.check()
    dt = time.perf_counter() - t0
    assert e.value.status == 6, str(e.value)  # FMM_ERR_TIMEOUT
    sites = int(str(e.value).rsplit("0x", 1)[1].rstrip(")"), 16)
    assert sites & ((1 << W_MMA_A) | (1 << W_EPI)), str(e.value)
    assert 1.5 < dt < 30.0  # the 2 s limit ran out once, then every CTA gave up
    plan.check()  # the flag was cleared

    phi = plan.solve(rho)
    torch.cuda.synchronize()
    plan.check()
    ref = orc.fmm(rho32.astype(np.float64), 4, 6)["phi"]
    err = float(np.linalg.norm(phi.double().cpu().numpy() - ref) / np.linalg.norm(ref))
    assert err <= 1e-5
    plan.close()


def test_debug_timeout_needs_a_prefix_m2l():
    plan = fmm.FMMPlan((64, 64, 64), 6, 4, "fp32")  # no tensor-core level
    with pytest.raises(fmm.FMMError):
        plan.debug_timeout()
    plan.close()
