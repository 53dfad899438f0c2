"""Analytic acceleration (accel = "analytic": the gradient of the leaf local
expansions plus the near-field pair forces; with the paper's final stage the
gradient of the leaf interaction list's M2P at the cell centres too) against
the oracle's analytic force, at every precision, on tensor cores and CUDA
cores.

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


def solve(rho, b, p, prec, dx=1.0, G=1.0, final_stage="m2l", m2p_schedule=None):
    nz, ny, nx = rho.shape
    plan = fmm.FMMPlan((nx, ny, nz), p, b, prec, dx=dx, G=G, accel="analytic", final_stage=final_stage)
    if m2p_schedule is not None:
        plan.set_tc_schedule("m2p", m2p_schedule)
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


def _adjoint(gphi, ga, b, p, prec, dx, G, final_stage="m2l"):
    nz, ny, nx = (gphi if gphi is not None else ga[0]).shape
    plan = fmm.FMMPlan((nx, ny, nz), p, b, prec, dx=dx, G=G, accel="analytic", final_stage=final_stage)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda().to(plan.dtype)  # noqa: E731
    g = plan.solve_adjoint(grad_phi=t(gphi) if gphi is not None else None, grad_accel=t(ga) if ga is not None else None)
    torch.cuda.synchronize()
    plan.check()
    out = g.double().cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3"])
def test_adjoint_of_the_analytic_force_matches_oracle(orc, prec):
    """grad_rho of <g_phi, phi> + <g_a, accel> with accel the analytic force:
    the GPU's transposed pipeline (dipole P2M sources for the force's L2P
    gradient, the near pair forces transposed into the same contraction as
    the potential's) against the oracle's explicit transpose chain."""
    rng = np.random.default_rng(31)
    shape, b, p, dx, G = (48, 32, 40), 4, 6, 0.3, 1.7
    gphi = rng.standard_normal(shape[::-1])
    ga = rng.standard_normal((3,) + shape[::-1])
    ref = orc.adjoint(gphi, ga, b, p, dx=dx, G=G, analytic=True)
    got = _adjoint(gphi, ga, b, p, prec, dx, G)
    err = rel(got, ref)
    print(f"{prec}: adjoint of the analytic force, rel err {err:.2e}")
    assert err <= {"fp64": 1e-10, "fp32": 1e-5, "bf16x3": 1e-5}[prec]
    # the force part alone
    ref_f = orc.adjoint(np.zeros(shape[::-1]), ga, b, p, dx=dx, G=G, analytic=True)
    got_f = _adjoint(None, ga, b, p, prec, dx, G)
    assert rel(got_f, ref_f) <= {"fp64": 1e-10, "fp32": 1e-5, "bf16x3": 1e-5}[prec]


@pytest.mark.parametrize("leaf", [2, 8])
def test_adjoint_of_the_analytic_force_other_leaf_sizes(orc, leaf):
    rng = np.random.default_rng(leaf)
    shape, p = (32, 24, 40), 4
    gphi = rng.standard_normal(shape[::-1])
    ga = rng.standard_normal((3,) + shape[::-1])
    ref = orc.adjoint(gphi, ga, leaf, p, analytic=True)
    assert rel(_adjoint(gphi, ga, leaf, p, "fp64", 1.0, 1.0), ref) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_adjoint_of_the_analytic_force_with_m2p_is_its_transpose(prec):
    """Final stage M2P: <g_phi, phi(rho)> + <g_a, accel(rho)> equals
    <adjoint(g_phi, g_a), rho>, the forward solves being the ones held to
    the oracle in test_analytic_accel_m2p_*; FP64 to rounding, bf16x3 to the
    split products' error."""
    rng = np.random.default_rng(5)
    shape, b, p, dx, G = (40, 32, 48), 4, 6, 0.4, 1.3
    rho = rng.standard_normal(shape[::-1])
    gphi = rng.standard_normal(shape[::-1])
    ga = rng.standard_normal((3,) + shape[::-1])
    phi, acc = solve(rho, b, p, prec, dx=dx, G=G, final_stage="m2p")
    lhs = np.vdot(gphi, phi) + np.vdot(ga, acc)
    at = _adjoint(gphi, ga, b, p, prec, dx, G, final_stage="m2p")
    rhs = np.vdot(at, rho)
    scale = np.abs(gphi).sum() * np.abs(phi).max() + np.abs(ga).sum() * np.abs(acc).max()
    print(f"{prec} m2p: <g, A rho> {lhs:.12e}, <A^T g, rho> {rhs:.12e}")
    assert abs(lhs - rhs) <= {"fp64": 1e-12, "bf16x3": 1e-6}[prec] * scale


def _m2p_schedules(b, p, prec):
    """The tensor-core M2P schedules a plan of this kind has (None: CUDA cores)."""
    plan = fmm.FMMPlan((32, 32, 32), p, b, prec, accel="analytic", final_stage="m2p")
    cur, avail = plan.tc_schedule("m2p")
    plan.close()
    return sorted(avail) if cur is not None else [None]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "tf32"])
def test_analytic_accel_m2p_final_stage_matches_oracle(orc, prec):
    """The paper's final stage (Sec. 4) with the analytic force: the leaf
    interaction list's M2P gradients at the cell centres (derivative tensors
    one order above the multipoles), on every M2P schedule the plan has."""
    rho = inputs.lognormal((64, 48, 80), seed=13).astype(np.float64)
    ref = orc.fmm_accel(rho, 4, 6, dx=0.5, G=2.0, final_stage="m2p")
    ref_phi = orc.fmm_m2p(rho, 4, 6, dx=0.5, G=2.0)
    tol = {"fp64": 1e-9, "fp32": 1e-5, "bf16x3": 1e-5, "tf32": 1e-3}[prec]
    for sched in _m2p_schedules(4, 6, prec):
        phi, acc = solve(rho, 4, 6, prec, dx=0.5, G=2.0, final_stage="m2p", m2p_schedule=sched)
        err, perr = rel(acc, ref), rel(phi, ref_phi)
        print(f"{prec} m2p ({sched}): analytic accel rel err {err:.2e}, phi {perr:.2e}")
        assert err <= tol, sched
        assert perr <= {"fp64": 1e-10, "fp32": 1e-5, "bf16x3": 1e-5, "tf32": 1e-3}[prec], sched


@pytest.mark.parametrize("leaf", [2, 8])
def test_analytic_accel_m2p_other_leaf_sizes(orc, leaf):
    rho = inputs.gaussian_blobs((32, 48, 40), seed=6)
    ref = orc.fmm_accel(rho, leaf, 4, final_stage="m2p")
    for prec in ("fp64", "bf16x3"):
        _, acc = solve(rho, leaf, 4, prec, final_stage="m2p")
        err = rel(acc, ref)
        print(f"leaf {leaf} {prec} m2p: analytic accel rel err {err:.2e}")
        assert err <= {"fp64": 1e-9, "bf16x3": 1e-5}[prec], (leaf, prec)
