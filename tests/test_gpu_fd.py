"""The force stencil (App. C) alone: the oracle's 5-point stencil applied to
the GPU's own potential must give the GPU's acceleration to FP32 rounding.
Shapes cover the vectorised path (nx % 4 == 0: full and partial 128-cell
tiles, narrow grids, partial z chunks) and the scalar one (nx % 4 == 2)."""
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


@pytest.mark.parametrize("shape,leaf", [((132, 20, 44), 4), ((36, 24, 72), 4), ((256, 8, 40), 8),
                                        ((38, 22, 18), 2), ((8, 8, 8), 4)])
def test_stencil_on_the_gpu_potential(orc, shape, leaf):
    nx, ny, nz = shape
    rho = inputs.gaussian_blobs(shape, seed=13).astype(np.float32)
    dx = 0.37
    plan = fmm.FMMPlan(shape, 4, leaf, "fp32", dx=dx)
    phi, acc = plan.solve(torch.from_numpy(rho).cuda(), accel=True)
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    phi64 = phi.double().cpu().numpy()
    ref = orc.fd_accel(phi64, dx=dx)
    got = acc.double().cpu().numpy()
    # FP32 stencil on FP32 values: the weights' absolute sum (1.5) times a few
    # ulps of |phi|, over dx (differences of nearby potentials cancel)
    bound = 1.5 * 4 * 2.0 ** -24 * np.max(np.abs(phi64)) / dx
    err = np.max(np.abs(got - ref))
    print(f"{shape} leaf {leaf}: max |accel - FD(phi)| = {err:.2e} (bound {bound:.2e})")
    assert err <= bound
