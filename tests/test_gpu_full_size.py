"""Dense parity at the benchmark size: 512^3 cells, leaf 4^3, the lognormal
field, orders 6 and 8, the bf16x3 tensor-core precision and FP32 plain,
against the FP64 oracle's sampled solve (oracle_fmm_sample: the same tree,
interaction lists and operators, evaluated at the chosen cells only).

The cells (2048 + 14) are whole x-rows chosen where the kernels' tiles and
the domain's edges are:
  * y = 127 | z = 255 and y = 128 | z = 256: the rows on both sides of the
    planes where the tensor-core M2L tiles of the leaf level meet (tiles of
    8 x 16 x 1 parents: every 128 cells in y, every 8 cells in z) and of the
    near-field tiles (8 x 16 x 1 leaf boxes: every 64 cells in y, 4 in z);
  * y = 0 | z = 0 and y = 511 | z = 511: rows along edges of the domain,
    where the activation boxes reach past it and are zero-filled;
  * the eight corners and six face centres.
A whole row spans every x tile boundary (8 parents = 64 cells).

Bounds: relative L2 <= 1e-5 (the metric's bound) and max |dphi| / max |phi|
<= 1e-5 (phi is smooth and positive-definite in sign here, so its maximum
norm and its L2 norm are within a small factor of each other; the errors of
the truncated split products are spread evenly, not concentrated at edges).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2606_13793_gb300 as fmm  # noqa: E402
from paper_2606_13793_gb300 import _build, inputs  # noqa: E402

N = 512


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    assert torch.cuda.is_available()


def dense_cells(n):
    rows = [(n // 4 - 1, n // 2 - 1), (n // 4, n // 2), (0, 0), (n - 1, n - 1)]
    x = np.arange(n)
    cells = [z * n * n + y * n + x for y, z in rows]
    corners = [z * n * n + y * n + xx for z in (0, n - 1) for y in (0, n - 1) for xx in (0, n - 1)]
    h = n // 2
    faces = [h * n * n + h * n + 0, h * n * n + h * n + n - 1, h * n * n + 0 * n + h, h * n * n + (n - 1) * n + h,
             0 * n * n + h * n + h, (n - 1) * n * n + h * n + h]
    return np.concatenate(cells + [np.array(corners + faces)]).astype(np.int64)


@pytest.fixture(scope="module")
def field():
    return inputs.lognormal(N, seed=2606)


_refs = {}


@pytest.fixture(scope="module")
def oracle_ref(orc, field):
    def get(p):
        if p not in _refs:
            cells = dense_cells(N)
            _refs[p] = (cells, orc.fmm_sample(field.astype(np.float64), 4, p, cells, dx=1.0 / N))
        return _refs[p]
    return get


@pytest.mark.parametrize("p", [6, 8])
@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_full_size_dense_rows(oracle_ref, field, p, prec):
    cells, ref = oracle_ref(p)
    plan = fmm.FMMPlan((N, N, N), p, 4, prec, dx=1.0 / N)
    plan.autotune()
    phi = plan.solve(torch.from_numpy(field).cuda())
    torch.cuda.synchronize()
    plan.check()
    got = phi.reshape(-1)[torch.from_numpy(cells).cuda()].double().cpu().numpy()
    plan.close()
    del phi
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    mx = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    worst = int(cells[np.argmax(np.abs(got - ref))])
    print(f"512^3 p={p} {prec}: {cells.size} cells, rel L2 {rel:.3e}, max|d|/max|phi| {mx:.3e} "
          f"(worst cell x={worst % N} y={worst // N % N} z={worst // N // N})")
    assert rel <= 1e-5
    assert mx <= 1e-5
