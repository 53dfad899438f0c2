"""mult_order < order (the paper keeps multipoles to order 2 and locals to
order 3, Sec. 2.1 and 2.3) against the oracle's separate-order solve, at
every precision and with either final stage, including the paper's own
configuration: order 3, multipoles to 2, final-stage M2P, leaf boxes of 2
cells.  Tolerances as for the symmetric solve (FP64 1e-10, FP32 and bf16x3
1e-5, TF32 1e-3)."""
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
    plan = fmm.FMMPlan((nx, ny, nz), p, b, prec, accel=False, **kw)
    r = torch.from_numpy(np.ascontiguousarray(rho)).cuda().to(plan.dtype)
    phi = plan.solve(r)
    torch.cuda.synchronize()
    plan.check()
    out = phi.double().cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "tf32"])
@pytest.mark.parametrize("p", [4, 6])
def test_reduced_multipole_order_matches_oracle(orc, prec, p):
    rho = inputs.lognormal((64, 48, 80), seed=21).astype(np.float64)
    ref = orc.fmm_orders(rho, 4, p, p - 1, p)
    err = rel(solve(rho, 4, p, prec, mult_order=p - 1), ref)
    print(f"p={p} mult_order={p - 1} {prec}: {err:.2e}")
    assert err <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3"])
def test_papers_configuration(orc, prec):
    """Order 3, multipoles to 2, final-stage M2P, leaf 2."""
    rho = inputs.plummer((32, 48, 64), seed=6).astype(np.float64)
    ref = orc.fmm_orders(rho, 2, 3, 2, 3, "m2p")
    err = rel(solve(rho, 2, 3, prec, mult_order=2, final_stage="m2p"), ref)
    print(f"paper's configuration {prec}: {err:.2e}")
    assert err <= TOL[prec]


def test_full_mult_order_is_the_default():
    rho = torch.from_numpy(inputs.lognormal(64, seed=2)).cuda()
    out = []
    for mo in (None, 6, 9):
        plan = fmm.FMMPlan((64, 64, 64), 6, 4, "bf16x3", accel=False, mult_order=mo)
        out.append(plan.solve(rho))
        torch.cuda.synchronize()
        plan.close()
    assert torch.equal(out[0], out[1]) and torch.equal(out[0], out[2])


def test_adjoint_rejected_for_reduced_multipole_order():
    plan = fmm.FMMPlan((32, 32, 32), 4, 4, "fp32", mult_order=3)
    g = torch.zeros((32, 32, 32), device="cuda")
    with pytest.raises(fmm.FMMError, match="UNSUPPORTED"):
        plan.solve_adjoint(g)
    plan.close()
