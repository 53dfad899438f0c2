"""mult_order < order (the paper keeps multipoles to order 2 and locals to
order 3, Sec. 2.1 and 2.3) against the oracle's separate-order solve, at
every precision and with either final stage, including the paper's own
configuration: order 3, multipoles to 2, final-stage M2P, leaf boxes of 2
cells.  Tolerances as for the symmetric solve (FP64 1e-10, FP32 and bf16x3
1e-5, TF32 1e-3).  The adjoint runs the transposed operator (the two order
limits swapped)."""
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


@pytest.mark.parametrize("final_stage,b,p,mo", [("m2l", 4, 4, 3), ("m2l", 4, 6, 4), ("m2p", 2, 3, 2)])
def test_reduced_multipole_order_adjoint_transposes_the_oracle(orc, final_stage, b, p, mo):
    """The transpose of multipoles-to-mo (locals to p) is the operator with the
    limits swapped: <g, A rho> with the oracle's separate-order solve equals
    <A^T g, rho> from the GPU adjoint, FP64; the last case is the paper's
    configuration (its leaf level by the transpose of M2P)."""
    rng = np.random.default_rng(p * 10 + mo)
    shape = (24, 32, 40)
    nx, ny, nz = shape
    rho = rng.standard_normal((nz, ny, nx))
    g = rng.standard_normal((nz, ny, nx))
    lhs = float(np.sum(g * orc.fmm_orders(rho, b, p, mo, p, final_stage)))
    plan = fmm.FMMPlan(shape, p, b, "fp64", accel=False, mult_order=mo, final_stage=final_stage)
    grad = plan.solve_adjoint(torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    plan.check()
    rhs = float(np.sum(grad.cpu().numpy() * rho))
    plan.close()
    scale = np.linalg.norm(g) * np.linalg.norm(orc.fmm_orders(rho, b, p, mo, p, final_stage))
    print(f"{final_stage} p={p} mo={mo}: {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= 1e-12 * scale


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_reduced_multipole_order_adjoint_mixed(prec):
    rng = np.random.default_rng(8)
    shape = (32, 48, 40)
    nx, ny, nz = shape
    plan = fmm.FMMPlan(shape, 6, 4, prec, accel=False, mult_order=5)
    rho = torch.from_numpy(rng.standard_normal((nz, ny, nx)).astype(np.float32)).cuda()
    g = torch.from_numpy(rng.standard_normal((nz, ny, nx)).astype(np.float32)).cuda()
    phi = plan.solve(rho)
    grad = plan.solve_adjoint(g)
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    lhs = float(torch.sum(g.double() * phi.double()))
    rhs = float(torch.sum(grad.double() * rho.double()))
    scale = float(torch.linalg.vector_norm(g.double()) * torch.linalg.vector_norm(phi.double()))
    print(f"{prec}: {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= 1e-5 * scale
