"""The paper's final stage (final_stage = "m2p": the leaf interaction list
evaluated by M2P at the cell centres) against the oracle's M2P solve, on
tensor cores (bf16x3, TF32) and CUDA cores (FP32, FP64), at the parity
tolerances of the M2L path (FP64 1e-10, FP32 and bf16x3 1e-5, TF32 1e-3).
Its adjoint runs the transpose of the leaf M2P (P2L into the leaf locals)."""
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


def test_m2p_accepts_analytic_accel():
    """The analytic force with the paper's final stage is built (its parity
    with the oracle is in test_gpu_accel.py)."""
    plan = fmm.FMMPlan((32, 32, 32), 4, 4, "fp32", final_stage="m2p", accel="analytic")
    plan.close()


@pytest.mark.parametrize("shape,b,p", [((24, 16, 20), 4, 4), ((16, 24, 32), 2, 3), ((32, 32, 32), 8, 4)])
def test_m2p_adjoint_is_the_transpose_of_the_oracle(orc, shape, b, p):
    """The adjoint with the final-stage M2P (P2L into the leaf locals, then
    L2L and L2P): <g_phi, phi(rho)> + <g_a, a(rho)> of the oracle's M2P solve
    equals <adjoint(g), rho> on the GPU, FP64 (the third case has no parent
    far field at the leaf level)."""
    rng = np.random.default_rng(b * 10 + p)
    nx, ny, nz = shape
    dx, G = 0.5, 2.0
    rho = rng.standard_normal((nz, ny, nx))
    gphi = rng.standard_normal((nz, ny, nx))
    gacc = rng.standard_normal((3, nz, ny, nx))
    phi = orc.fmm_m2p(rho, b, p, dx=dx, G=G)
    acc = orc.fd_accel(phi, dx=dx)
    lhs = float(np.sum(gphi * phi) + np.sum(gacc * acc))
    plan = fmm.FMMPlan(shape, p, b, "fp64", dx=dx, G=G, final_stage="m2p")
    grad = plan.solve_adjoint(torch.from_numpy(gphi).cuda(), torch.from_numpy(gacc).cuda())
    torch.cuda.synchronize()
    plan.check()
    rhs = float(np.sum(grad.cpu().numpy() * rho))
    scale = np.linalg.norm(gphi) * np.linalg.norm(phi) + np.linalg.norm(gacc) * np.linalg.norm(acc)
    print(f"{shape} b={b} p={p}: |<g, A rho> - <A^T g, rho>| / scale = {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= 1e-12 * scale
    # a later forward solve is unaffected by the adjoint's use of the leaf locals
    r = torch.from_numpy(rho).cuda()
    a1 = plan.solve(r)
    plan.solve_adjoint(torch.from_numpy(gphi).cuda())
    a2 = plan.solve(r)
    torch.cuda.synchronize()
    assert torch.equal(a1, a2)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_m2p_adjoint_transposes_the_forward(prec):
    rng = np.random.default_rng(4)
    shape = (32, 48, 40)
    nx, ny, nz = shape
    plan = fmm.FMMPlan(shape, 6, 4, prec, final_stage="m2p")
    rho = torch.from_numpy(rng.standard_normal((nz, ny, nx)).astype(np.float32)).cuda()
    g = torch.from_numpy(rng.standard_normal((nz, ny, nx)).astype(np.float32)).cuda()
    phi, _ = plan.solve(rho, accel=True)
    grad = plan.solve_adjoint(g)
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    lhs = float(torch.sum(g.double() * phi.double()))
    rhs = float(torch.sum(grad.double() * rho.double()))
    scale = float(torch.linalg.vector_norm(g.double()) * torch.linalg.vector_norm(phi.double()))
    print(f"{prec}: {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= 1e-5 * scale
