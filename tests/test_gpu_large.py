"""1024^3 forward and backward (FP32, p = 6, leaf 4): the largest grid run.

Loss = 0.5 ||phi - phi_t||^2 with phi_t the potential of a second seeded
lognormal field; the backward pass is fmm_solve_adjoint through the autograd
Function.  The solve is linear, so the backward pass keeps no activations:
it re-runs the plan's kernels on dLoss/dphi (the only per-level state is the
plan's own workspace, reused).  Checked at sampled cells against the FP64
oracle: phi (1e-5), accel (FD tolerance 1e-4 * n / 256) and the gradient
(1e-4, the adjoint's bound).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2606_13793_gb300 as fmm  # noqa: E402
from paper_2606_13793_gb300 import _build, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    assert torch.cuda.is_available()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_forward_backward_1024(orc):
    n, p, b = 1024, 6, 4
    dx = 1.0 / n
    plan = fmm.FMMPlan((n, n, n), p, b, "fp32", dx=dx)
    with torch.no_grad():
        phit = plan.solve(torch.from_numpy(inputs.lognormal(n, seed=2607)).cuda())
    # torch builds its float64 reduction kernels on first use (seconds); do it
    # on a tiny tensor so the timings below are the solves'
    w = torch.ones(8, device="cuda")
    (0.5 * ((w - w) ** 2).sum(dtype=torch.float64)).item()
    rho_np = inputs.lognormal(n, seed=2606)
    rho = torch.from_numpy(rho_np).cuda().requires_grad_(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    phi, acc = fmm.FMMSolve.apply(rho, plan)
    ev[1].record()
    loss = 0.5 * ((phi - phit) ** 2).sum(dtype=torch.float64)
    loss.backward()
    ev[2].record()
    torch.cuda.synchronize()
    plan.check()
    print(f"1024^3 forward {ev[0].elapsed_time(ev[1]):.1f} ms, loss + backward {ev[1].elapsed_time(ev[2]):.1f} ms, "
          f"workspace {plan.workspace_bytes / 2**30:.1f} GiB")

    rng = np.random.default_rng(11)
    cells = rng.integers(0, n ** 3, 24)
    cells[:3] = [0, n ** 3 - 1, n // 2 * (n * n + n + 1)]
    idx = torch.from_numpy(cells).cuda()
    got_phi = phi.detach().reshape(-1)[idx].double().cpu().numpy()
    got_acc = acc.detach().reshape(3, -1)[:, idx].double().cpu().numpy().T
    got_grad = rho.grad.reshape(-1)[idx].double().cpu().numpy()
    g = (phi.detach() - phit).double().cpu().numpy()
    del phi, acc, phit, rho
    torch.cuda.empty_cache()

    ref_phi, ref_acc = orc.fmm_sample(rho_np.astype(np.float64), b, p, cells, dx=dx, accel=True)
    del rho_np
    assert rel_l2(got_phi, ref_phi) <= 1e-5
    assert rel_l2(got_acc, ref_acc) <= 1e-4 * n / 256
    # the operator is symmetric, so the adjoint of phi is the same solve of g
    ref_grad = orc.fmm_sample(g, b, p, cells, dx=dx)
    err = rel_l2(got_grad, ref_grad)
    print(f"gradient rel err at sampled cells {err:.2e}")
    assert err <= 1e-4
    plan.close()
