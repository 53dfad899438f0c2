"""Analytic acceleration (accel = "analytic": the gradient of the leaf local
expansions plus the near-field pair forces) against the oracle's analytic
force, at every precision, on tensor cores and CUDA cores.

Tolerances (relative L2 over all components): FP64 1e-10 (rounding order);
FP32 1e-5 (no stencil here, so the force carries the potential's relative
error rather than the stencil's amplification of it); bf16x3 1e-5, the
metric's bound (the split products are accurate to ~4e-6 of the sum of
|terms|; the tensor cores' truncating FP32 accumulation is bounded by the
near field's per-column accumulation segments at leaf 8); TF32 1e-3.
"""
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


def solve(rho, b, p, prec, dx=1.0, G=1.0):
    nz, ny, nx = rho.shape
    plan = fmm.FMMPlan((nx, ny, nz), p, b, prec, dx=dx, G=G, accel="analytic")
    r = torch.from_numpy(np.ascontiguousarray(rho)).cuda().to(plan.dtype)
    phi, acc = plan.solve(r, accel=True)
    torch.cuda.synchronize()
    plan.check()
    out = phi.double().cpu().numpy(), acc.double().cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "tf32"])
def test_analytic_accel_matches_oracle(orc, prec):
    rho = inputs.lognormal((64, 48, 80), seed=12).astype(np.float64)
    ref = orc.fmm_accel(rho, 4, 6, dx=0.5, G=2.0)
    ref_phi = orc.fmm(rho, 4, 6, dx=0.5, G=2.0)["phi"]
    phi, acc = solve(rho, 4, 6, prec, dx=0.5, G=2.0)
    err = rel(acc, ref)
    print(f"{prec}: analytic accel rel err {err:.2e}")
    assert err <= TOL[prec]
    assert rel(phi, ref_phi) <= {"fp64": 1e-10, "fp32": 1e-5, "bf16x3": 1e-5, "tf32": 1e-3}[prec]


@pytest.mark.parametrize("leaf", [2, 8])
def test_analytic_accel_other_leaf_sizes(orc, leaf):
    rho = inputs.gaussian_blobs((32, 48, 40), seed=2)
    ref = orc.fmm_accel(rho, leaf, 4)
    for prec in ("fp64", "bf16x3"):
        _, acc = solve(rho, leaf, 4, prec)
        err = rel(acc, ref)
        print(f"leaf {leaf} {prec}: analytic accel rel err {err:.2e}")
        assert err <= TOL[prec], (leaf, prec)


def test_analytic_accel_full_size_sampled(orc):
    n = 512
    rho = inputs.lognormal(n, seed=2606)
    plan = fmm.FMMPlan((n, n, n), 6, 4, "bf16x3", dx=1.0 / n, accel="analytic")
    _, acc = plan.solve(torch.from_numpy(rho).cuda(), accel=True)
    torch.cuda.synchronize()
    plan.check()
    rng = np.random.default_rng(3)
    cells = rng.integers(0, n ** 3, 24)
    cells[:2] = [n // 2 * (n * n + n + 1), 7 * n * n + 100 * n + 300]
    got = np.stack([acc[q].reshape(-1)[torch.from_numpy(cells).cuda()].double().cpu().numpy() for q in range(3)], 1)
    ref = orc.fmm_sample_accel(rho.astype(np.float64), 4, 6, cells, dx=1.0 / n)
    assert rel(got, ref) <= 1e-5
    plan.close()


def test_analytic_accel_adjoint_of_accel_is_rejected():
    plan = fmm.FMMPlan((32, 32, 32), 4, 4, "fp32", accel="analytic")
    g = torch.zeros(3, 32, 32, 32, device="cuda")
    with pytest.raises(fmm.FMMError) as e:
        plan.solve_adjoint(grad_accel=g)
    assert e.value.status == 2
    plan.close()
