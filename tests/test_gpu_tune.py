"""CUDA-core contraction variants and their autotuner.

Every variant (tile shape 0 = 4x4x4 rows, 1 and 2 = z-run register tiles,
3 = one column per lane; neighbour split 1 / 3 / 9 / 27) is forced on every M2L level off the tensor
cores and on the near field, and the solve is held to the oracle at the
precision's parity tolerance (FP64 1e-10, FP32 1e-5 relative L2 on phi).
The autotuner's picks must be valid variants and give the same answer.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2606_13793_gb300 as fmm  # noqa: E402
from paper_2606_13793_gb300 import _build, inputs  # noqa: E402

VARIANTS = [(0, 1), (0, 27), (1, 1), (1, 3), (1, 9), (2, 1), (2, 3), (2, 9), (3, 1), (3, 27)]
TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def case(orc):
    shape = (96, 64, 80)
    rho = inputs.plummer(shape, seed=21).astype(np.float64)
    return shape, rho, orc.fmm(rho, 4, 6, accel=True)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def force(plan, shape, dsplit):
    """Set the variant wherever it applies; returns how many contractions took it."""
    n = 0
    for lvl in list(range(2, plan.leaf_level + 1)) + [-1]:
        try:
            plan.set_tuning(lvl, shape, dsplit)
            n += 1
        except fmm.FMMError:
            pass
    return n


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_matches_oracle(case, prec, variant):
    shape, rho, ref = case
    plan = fmm.FMMPlan(shape, 6, 4, prec)
    took = force(plan, *variant)
    assert took >= 1
    r = torch.from_numpy(rho).cuda().to(plan.dtype)
    phi, acc = plan.solve(r, accel=True)
    torch.cuda.synchronize()
    plan.check()
    err = rel_l2(phi.double().cpu().numpy(), ref["phi"])
    print(f"{prec} variant {variant} on {took} contractions: phi rel err {err:.2e}")
    assert err <= TOL[prec]
    assert rel_l2(acc.double().cpu().numpy(), ref["accel"]) <= (1e-9 if prec == "fp64" else 1e-4)
    plan.close()


def test_variant_rejected_where_it_does_not_apply():
    plan = fmm.FMMPlan((64, 64, 64), 6, 4, "bf16x3", coarse="fp64")
    with pytest.raises(fmm.FMMError):
        plan.set_tuning(plan.leaf_level, 1, 1)  # a tensor-core level
    with pytest.raises(fmm.FMMError):
        plan.set_tuning(3, 1, 27)  # z-run tiles split 1, 3 or 9 ways
    with pytest.raises(fmm.FMMError):
        plan.set_tuning(3, 1, 1)  # FP64 levels of a tensor-core plan keep small-footprint tiles
    with pytest.raises(fmm.FMMError):
        plan.set_tuning(3, 4, 1)
    plan.set_tuning(3, 3, 27)
    assert plan.tuning(3) == (3, 27)
    plan.close()
    plan = fmm.FMMPlan((64, 64, 64), 6, 4, "bf16x3")  # FP32 coarse levels (default): z-run tiles apply
    plan.set_tuning(3, 1, 1)
    assert plan.tuning(3) == (1, 1)
    with pytest.raises(fmm.FMMError):
        plan.set_tuning(plan.leaf_level, 1, 1)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotune_picks_valid_variants(case, prec):
    shape, rho, ref = case
    plan = fmm.FMMPlan(shape, 6, 4, prec)
    plan.autotune()
    picks = {lvl: plan.tuning(lvl) for lvl in list(range(2, plan.leaf_level + 1)) + [-1]}
    print(prec, picks)
    for s, d in picks.values():
        assert (s, d) in VARIANTS
    r = torch.from_numpy(rho).cuda().to(plan.dtype)
    phi = plan.solve(r)
    torch.cuda.synchronize()
    plan.check()
    assert rel_l2(phi.double().cpu().numpy(), ref["phi"]) <= TOL[prec]
    # a second plan of the same shape takes the cached picks
    p2 = fmm.FMMPlan(shape, 6, 4, prec)
    p2.autotune()
    assert {lvl: p2.tuning(lvl) for lvl in picks} == picks
    assert p2.launches(True) == plan.launches(True)
    p2.close()
    plan.close()


@pytest.mark.parametrize("leaf", [2, 8])
def test_zrun_near_field_other_leaf_sizes(orc, leaf):
    shape = (64, 48, 32)
    rho = inputs.gaussian_blobs(shape, seed=8)
    ref = orc.fmm(rho, leaf, 4)
    for variant in [(1, 1), (2, 3)]:
        plan = fmm.FMMPlan(shape, 4, leaf, "fp64")
        plan.set_tuning(-1, *variant)
        phi = plan.solve(torch.from_numpy(rho).cuda())
        torch.cuda.synchronize()
        plan.check()
        assert rel_l2(phi.cpu().numpy(), ref["phi"]) <= 1e-10, (leaf, variant)
        plan.close()
