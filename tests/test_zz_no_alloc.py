"""fmm_solve_static: the solve for callers that cannot allocate device memory
(a latency-bound loop where cudaMalloc could synchronise the device, code under
a framework allocator that owns the memory budget, a plug-in that may not
allocate after start-up).  It has no plan and uses the library's fixed 16 MiB
static device array as its workspace.

Checked through the C ABI against the planned FP32 solve (fmm_solve), on two
calls in a row -- the second reuses the tables the first left in the static
array -- within the FP32 tolerance of the parity tests (1e-5 relative L2 on
phi, 1e-4 on accel), and against the FP64 oracle; free device memory is
unchanged across repeated calls (same and changed shapes); output tensors of
the wrong shape, type, layout or device are rejected before the call.  This
file is collected last on purpose, and it passes alone in a fresh process as
well as after the other tests.
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
    a, b = a.double().cpu(), b.double().cpu()
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def planned(rho, order, leaf, dx):
    nz, ny, nx = rho.shape
    plan = fmm.FMMPlan((nx, ny, nz), order, leaf, "fp32", dx=dx)
    phi, acc = plan.solve(rho, accel=True)
    torch.cuda.synchronize()
    plan.close()
    return phi, acc


def test_static_solve_matches_planned_solve_twice():
    n, order, leaf, dx = 64, 6, 4, 1.0 / 64
    phi = torch.empty(n, n, n, device="cuda")
    acc = torch.empty(3, n, n, n, device="cuda")
    for seed in (2606, 2607):  # two calls in a row, same shape
        rho = torch.from_numpy(inputs.lognormal(n, seed=seed)).cuda()
        fmm.solve_static(rho, order, leaf, dx=dx, accel=True, phi_out=phi, accel_out=acc)
        torch.cuda.synchronize()
        ref_phi, ref_acc = planned(rho, order, leaf, dx)
        assert rel_l2(phi, ref_phi) <= 1e-5
        assert rel_l2(acc, ref_acc) <= 1e-4


def test_static_solve_other_shape_then_back():
    """A different grid rebuilds the tables in the static array; going back
    rebuilds them again.  Both answers match the planned solve."""
    for shape in ((32, 48, 40), (64, 64, 64)):
        nx, ny, nz = shape
        rho = torch.from_numpy(inputs.plummer(shape, seed=3)).cuda()
        phi = fmm.solve_static(rho, 4, 4)
        torch.cuda.synchronize()
        ref, _ = planned(rho, 4, 4, 1.0)
        assert rel_l2(phi, ref) <= 1e-5


def test_static_solve_rejects_too_large():
    rho = torch.zeros(128, 128, 128, device="cuda")
    with pytest.raises(fmm.FMMError) as e:
        fmm.solve_static(rho, 6, 4)
    assert e.value.status == 1 and "static" in str(e.value)
    with pytest.raises(fmm.FMMError):
        fmm.solve_static(torch.zeros(32, 32, 32, device="cuda"), 7, 4)


def test_static_solve_matches_oracle(orc):
    n, order, leaf = 32, 6, 4
    rho = inputs.lognormal(n, seed=41)
    ref = orc.fmm(rho.astype(np.float64), leaf, order, accel=True)
    phi, acc = fmm.solve_static(torch.from_numpy(rho).cuda(), order, leaf, accel=True)
    torch.cuda.synchronize()
    assert rel_l2(phi, torch.from_numpy(ref["phi"])) <= 1e-5
    assert rel_l2(acc, torch.from_numpy(ref["accel"])) <= 1e-4


def test_static_solve_allocates_no_device_memory():
    """Free device memory (cudaMemGetInfo: every allocator of the process,
    not only torch's) stays the same over repeated calls with caller-owned
    outputs, for an unchanged shape and for changed shapes."""
    shapes = [(32, 32, 32), (32, 32, 32), (24, 40, 32), (32, 32, 32)]
    bufs = []
    for nz, ny, nx in shapes:
        rho = torch.from_numpy(inputs.plummer((nx, ny, nz), seed=9)).cuda()
        bufs.append((rho, torch.empty_like(rho), torch.empty((3, nz, ny, nx), device="cuda")))
    fmm.solve_static(bufs[0][0], 4, 4, accel=True, phi_out=bufs[0][1], accel_out=bufs[0][2])  # warm-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for rho, phi, acc in bufs:
            fmm.solve_static(rho, 4, 4, accel=True, phi_out=phi, accel_out=acc)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_solve_rejects_bad_outputs():
    rho = torch.zeros(32, 32, 32, device="cuda")
    with pytest.raises(ValueError):
        fmm.solve_static(rho, 4, 4, phi_out=torch.empty(32, 32, 16, device="cuda"))
    with pytest.raises(ValueError):
        fmm.solve_static(rho, 4, 4, accel=True, accel_out=torch.empty(3, 32, 32, 31, device="cuda"))
    with pytest.raises(TypeError):
        fmm.solve_static(rho, 4, 4, phi_out=torch.empty(32, 32, 32, device="cuda", dtype=torch.float64))
    with pytest.raises(TypeError):
        fmm.solve_static(rho, 4, 4, phi_out=torch.empty(32, 32, 32))  # host memory
    with pytest.raises(ValueError):
        fmm.solve_static(rho, 4, 4, phi_out=torch.empty(32, 32, 64, device="cuda")[:, :, ::2])
