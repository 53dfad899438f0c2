"""The paper's final stage (final_stage = "m2p": the leaf interaction list
evaluated by M2P at the cell centres) against the oracle's M2P solve, on
tensor cores (bf16x3, TF32) and CUDA cores (FP32, FP64), at the parity
tolerances of the M2L path (FP64 1e-10, FP32 and bf16x3 1e-5, TF32 1e-3)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2606_13793_gb300 as fmm  # noqa: E402
from paper_2606_13793_gb300 import _build, inputs  # noqa: E402

TOL = {"fp64": 1e-10, "fp32": 1e-5, "bf16x3": 1e-5, "tf32": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    assert torch.cuda.is_available()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def solve(rho, b, p, prec, **kw):
    nz, ny, nx = rho.shape
    plan = fmm.FMMPlan((nx, ny, nz), p, b, prec, final_stage="m2p", **kw)
    phi = plan.solve(torch.from_numpy(np.ascontiguousarray(rho)).cuda().to(plan.dtype))
    torch.cuda.synchronize()
    plan.check()
    out = phi.double().cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "tf32"])
def test_m2p_matches_oracle(orc, prec):
    rho = inputs.lognormal((64, 48, 80), seed=13).astype(np.float64)
    ref = orc.fmm_m2p(rho, 4, 6, dx=0.5, G=2.0)
    err = rel(solve(rho, 4, 6, prec, dx=0.5, G=2.0), ref)
    print(f"{prec}: final-stage M2P phi rel err {err:.2e}")
    assert err <= TOL[prec]


@pytest.mark.parametrize("leaf", [2, 8])
def test_m2p_other_leaf_sizes(orc, leaf):
    rho = inputs.plummer((32, 48, 64), seed=6).astype(np.float64)
    ref = orc.fmm_m2p(rho, leaf, 4)
    for prec in ("fp64", "bf16x3"):
        assert rel(solve(rho, leaf, 4, prec), ref) <= TOL[prec], (leaf, prec)


def test_m2p_more_accurate_than_m2l_l2p(orc):
    """Against the direct sum, the final-stage M2P beats M2L + L2P at equal order."""
    rho = inputs.gaussian_blobs(32, seed=5)
    d = orc.direct(rho)
    plan = fmm.FMMPlan((32, 32, 32), 4, 4, "fp64")
    m2l = plan.solve(torch.from_numpy(rho).cuda()).cpu().numpy()
    plan.close()
    assert rel(solve(rho, 4, 4, "fp64"), d) < rel(m2l, d)


def test_m2p_rejects_adjoint_and_analytic_accel():
    plan = fmm.FMMPlan((32, 32, 32), 4, 4, "fp32", final_stage="m2p")
    with pytest.raises(fmm.FMMError) as e:
        plan.solve_adjoint(torch.zeros(32, 32, 32, device="cuda"))
    assert e.value.status == 2
    plan.close()
    with pytest.raises(fmm.FMMError):
        fmm.FMMPlan((32, 32, 32), 4, 4, "fp32", final_stage="m2p", accel="analytic")
