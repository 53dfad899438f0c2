"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 over all cells, from the arithmetic of each mode):
  FP64         phi <= 1e-10, accel <= 1e-9   (rounding-order differences only)
  FP32 plain   phi <= 1e-5                   (FP32 unit roundoff 6e-8 times the
                                              depth of the sums, with margin)
               accel <= acc_tol(n)           the stencil differences phi over
                                              one cell: an error e in phi becomes
                                              about 1.5 e |phi| / |dphi/di| ~
                                              0.4 n e relative in accel, so with
                                              e <= 1e-6: 1e-4 * max(1, n / 256)
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


def acc_tol(n):
    return 1e-4 * max(1.0, n / 256.0)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def gpu_solve(rho, b, p, precision, dx=1.0, G=1.0, accel=True):
    nz, ny, nx = rho.shape
    plan = fmm.FMMPlan((nx, ny, nz), p, b, precision, dx=dx, G=G)
    dt = torch.float64 if precision == "fp64" else torch.float32
    r = torch.from_numpy(np.ascontiguousarray(rho)).to(device="cuda", dtype=dt)
    if accel:
        phi, acc = plan.solve(r, accel=True)
    else:
        phi, acc = plan.solve(r), None
    torch.cuda.synchronize()
    plan.check()
    out = phi.double().cpu().numpy(), (acc.double().cpu().numpy() if acc is not None else None)
    plan.close()
    return out


FP64_CASES = [
    # (shape (nx, ny, nz), leaf, order)
    ((32, 32, 32), 4, 4),    # the 32^3 FP64 configuration (8^3 leaves)
    ((8, 8, 8), 4, 4),       # two leaves per axis: no M2L at all
    ((4, 4, 4), 4, 2),       # a single leaf box
    ((4, 4, 4), 2, 3),       # leaf 2
    ((24, 20, 28), 4, 5),    # ragged, non-power-of-two extents (phantom boxes)
    ((16, 32, 8), 2, 4),
    ((64, 16, 16), 8, 3),    # leaf 8
    ((40, 24, 32), 4, 8),    # maximum order
    ((32, 32, 32), 4, 0),    # monopole only
]


@pytest.mark.parametrize("shape,b,p", FP64_CASES)
def test_fp64_matches_oracle(orc, shape, b, p):
    rho = inputs.gaussian_blobs(shape, seed=2606 + p)
    ref = orc.fmm(rho, b, p, dx=0.03125, G=1.0, accel=True)
    phi, acc = gpu_solve(rho, b, p, "fp64", dx=0.03125, G=1.0)
    assert rel_l2(phi, ref["phi"]) <= 1e-10
    assert rel_l2(acc, ref["accel"]) <= 1e-9


def test_fp64_config_against_direct_sum(orc):
    """32^3, p=4, leaf 4: the GPU solve matches the oracle and sits as close
    to the O(N^2) direct sum as the oracle does."""
    rho = inputs.gaussian_blobs(32, seed=2606)
    direct = orc.direct(rho)
    phi, _ = gpu_solve(rho, 4, 4, "fp64")
    ref = orc.fmm(rho, 4, 4)["phi"]
    assert rel_l2(phi, ref) <= 1e-10
    assert abs(rel_l2(phi, direct) - rel_l2(ref, direct)) <= 1e-9


def test_fp64_levels_match_oracle(orc):
    shape, b, p = (32, 24, 40), 4, 5
    rho = inputs.gaussian_blobs(shape, seed=77)
    nz, ny, nx = rho.shape
    plan = fmm.FMMPlan((nx, ny, nz), p, b, "fp64")
    plan.solve(torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    L = plan.leaf_level
    for lvl in range(2, L + 1):
        ref = orc.fmm(rho, b, p, export_level=lvl)
        for what in ("M", "L"):
            got = plan.debug_level(what, lvl)
            np.testing.assert_allclose(got, ref[what], rtol=1e-10, atol=1e-11 * np.abs(ref[what]).max(),
                                       err_msg=f"{what} level {lvl}")
    plan.close()


def test_fp32_matches_oracle(orc):
    rho = inputs.lognormal(64, seed=2606).astype(np.float64)
    ref = orc.fmm(rho, 4, 6, accel=True)
    phi, acc = gpu_solve(rho.astype(np.float32), 4, 6, "fp32")
    assert rel_l2(phi, ref["phi"]) <= 1e-5
    assert rel_l2(acc, ref["accel"]) <= 1e-4


def test_fp32_ragged_matches_oracle(orc):
    rho = inputs.plummer((96, 64, 80), seed=5).astype(np.float64)
    ref = orc.fmm(rho, 4, 6, accel=True)
    phi, acc = gpu_solve(rho.astype(np.float32), 4, 6, "fp32")
    assert rel_l2(phi, ref["phi"]) <= 1e-5
    assert rel_l2(acc, ref["accel"]) <= 1e-4


@pytest.mark.parametrize("n", [256, 512])
def test_fp32_full_size_sampled(orc, n):
    """The benchmark sizes (256^3 and 512^3, p=6, leaf 4, lognormal field):
    sampled cells, including edges and the zeroed margin, against the
    oracle's per-cell evaluation."""
    rho32 = inputs.lognormal(n, seed=2606)
    phi, acc = gpu_solve(rho32, 4, 6, "fp32", dx=1.0 / n)
    rng = np.random.default_rng(1)
    cells = rng.integers(0, n ** 3, 48)
    cells[:6] = [0, n ** 3 - 1, n // 2 * (n * n + n + 1), n - 1, n * n * (n - 1), (n // 2) * n * n + 3 * n + 7]
    ref_phi, ref_acc = orc.fmm_sample(rho32.astype(np.float64), 4, 6, cells, dx=1.0 / n, accel=True)
    assert rel_l2(phi.ravel()[cells], ref_phi) <= 1e-5
    got_acc = np.stack([acc[q].ravel()[cells] for q in range(3)], 1)
    assert rel_l2(got_acc, ref_acc) <= acc_tol(n)


def test_adjoint_fp64_matches_oracle(orc):
    rng = np.random.default_rng(3)
    shape, b, p, dx, G = (24, 16, 20), 4, 4, 0.5, 2.0
    nx, ny, nz = shape
    gphi = rng.standard_normal((nz, ny, nx))
    gacc = rng.standard_normal((3, nz, ny, nx))
    ref = orc.adjoint(gphi, gacc, b, p, dx=dx, G=G)
    plan = fmm.FMMPlan(shape, p, b, "fp64", dx=dx, G=G)
    g = plan.solve_adjoint(torch.from_numpy(gphi).cuda(), torch.from_numpy(gacc).cuda())
    torch.cuda.synchronize()
    assert rel_l2(g.cpu().numpy(), ref) <= 1e-10
    plan.close()


def test_adjoint_fp32_matches_oracle(orc):
    rng = np.random.default_rng(4)
    shape, b, p = (32, 32, 32), 4, 6
    gphi = rng.standard_normal((32, 32, 32))
    gacc = rng.standard_normal((3, 32, 32, 32))
    ref = orc.adjoint(gphi, gacc, b, p, dx=1 / 32)
    plan = fmm.FMMPlan(shape, p, b, "fp32", dx=1 / 32)
    g = plan.solve_adjoint(torch.from_numpy(gphi).float().cuda(), torch.from_numpy(gacc).float().cuda())
    torch.cuda.synchronize()
    assert rel_l2(g.cpu().numpy(), ref) <= 1e-5
    plan.close()


def test_autograd_finite_differences():
    """Loss 0.5 ||phi(rho) - phi_t||^2 + 0.5 ||accel||^2 at 32^3: the
    backward pass matches central differences (eps 1e-3, 64 seeded cells)
    to 1e-4 relative.  FP64 solve, FP64 loss accumulation."""
    n, p = 32, 6
    rho = torch.from_numpy(inputs.lognormal(n, seed=1).astype(np.float64)).cuda()
    tgt = torch.from_numpy(inputs.lognormal(n, seed=2).astype(np.float64)).cuda()
    plan = fmm.FMMPlan((n, n, n), p, 4, "fp64", dx=1 / n)
    phi_t, _ = plan.solve(tgt, accel=True)

    def loss(r):
        phi, acc = fmm.FMMSolve.apply(r, plan)
        return 0.5 * ((phi - phi_t) ** 2).sum() + 0.5 * (acc ** 2).sum()

    x = rho.clone().requires_grad_(True)
    L = loss(x)
    L.backward()
    grad = x.grad.detach()
    rng = np.random.default_rng(64)
    cells = rng.integers(0, n ** 3, 64)
    eps = 1e-3
    flat = rho.view(-1)
    for c in cells:
        xp = flat.clone()
        xp[c] += eps
        xm = flat.clone()
        xm[c] -= eps
        with torch.no_grad():
            fd = (loss(xp.view(n, n, n)) - loss(xm.view(n, n, n))) / (2 * eps)
        g = grad.view(-1)[c]
        assert abs(float(fd - g)) <= 1e-4 * max(abs(float(g)), 1e-12)
    plan.close()


def test_nonfinite_input_is_reported():
    plan = fmm.FMMPlan((16, 16, 16), 4, 4, "fp32")
    rho = torch.ones(16, 16, 16, device="cuda")
    rho[3, 4, 5] = float("nan")
    plan.solve(rho)
    with pytest.raises(fmm.FMMError) as e:
        plan.check()
    assert e.value.status == 5
    plan.solve(torch.ones(16, 16, 16, device="cuda"))
    plan.check()  # cleared
    plan.close()


def test_deterministic_and_host_path():
    rho32 = inputs.lognormal(64, seed=9)
    plan = fmm.FMMPlan((64, 64, 64), 6, 4, "fp32")
    r = torch.from_numpy(rho32).cuda()
    a, aa = plan.solve(r, accel=True)
    b, bb = plan.solve(r, accel=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(aa, bb)
    phi_h = np.zeros_like(rho32)
    acc_h = np.zeros((3,) + rho32.shape, np.float32)
    plan.solve_host(rho32, phi_h, acc_h)
    assert np.array_equal(phi_h, a.cpu().numpy()) and np.array_equal(acc_h, aa.cpu().numpy())
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_host_many_equals_device_solves(precision):
    """fmm_solve_host_many (uploads and downloads on their own streams beside
    the solves, two staging sets): every field bit-equal to its device
    solve, with pinned and pageable buffers, a repeated input, one field
    (one staging set), no accel, none at all, and fmm_solve_host after it."""
    shape = (64, 48, 32)
    plan = fmm.FMMPlan(shape, 6, 4, precision)
    rhos = [inputs.plummer(shape, seed=40 + i) for i in range(4)]
    rhos.append(rhos[1])  # the same input buffer twice
    want = [plan.solve(torch.from_numpy(r).cuda(), accel=True) for r in rhos]
    want = [(a.cpu().numpy(), g.cpu().numpy()) for a, g in want]
    pin = [torch.from_numpy(r).pin_memory() for r in rhos]
    phis = [torch.empty(r.shape, dtype=torch.float32).pin_memory() for r in rhos]
    accs = [torch.empty((3,) + r.shape, dtype=torch.float32).pin_memory() for r in rhos]
    def same(x, y):  # FP32: the solve is deterministic; bf16x3 held to 1e-6 of the field's scale
        if precision == "fp32":
            return np.array_equal(x, y)
        return np.max(np.abs(x - y)) <= 1e-6 * np.max(np.abs(y))

    plan.solve_host_many(pin, phis, accs)
    for i, (a, g) in enumerate(want):
        assert same(phis[i].numpy(), a), i
        assert same(accs[i].numpy(), g), i
    # pageable numpy buffers, no accel, repeated twice over
    out = [np.zeros_like(r) for r in rhos[:3]]
    plan.solve_host_many(rhos[:3], out)
    plan.solve_host_many(rhos[:3], out)
    for i in range(3):
        assert same(out[i], want[i][0]), i
    one_phi, one_acc = np.zeros_like(rhos[2]), np.zeros((3,) + rhos[2].shape, np.float32)
    plan.solve_host_many([rhos[2]], [one_phi], [one_acc])
    assert same(one_phi, want[2][0]) and same(one_acc, want[2][1])
    plan.solve_host_many([], [])
    h_phi, h_acc = np.zeros_like(rhos[0]), np.zeros((3,) + rhos[0].shape, np.float32)
    plan.solve_host(rhos[0], h_phi, h_acc)
    assert same(h_phi, want[0][0]) and same(h_acc, want[0][1])
    with pytest.raises(ValueError):
        plan.solve_host_many(rhos[:2], out[:1])
    with pytest.raises(ValueError):
        plan.solve_host_many([rhos[0][:16]], [out[0]])
    plan.close()


def test_bad_arguments_raise():
    plan = fmm.FMMPlan((16, 16, 16), 4, 4, "fp32")
    with pytest.raises(ValueError):
        plan.solve(torch.ones(8, 16, 16, device="cuda"))
    with pytest.raises(TypeError):
        plan.solve(torch.ones(16, 16, 16, device="cuda", dtype=torch.float64))
    plan.close()
    with pytest.raises(fmm.FMMError):
        fmm.FMMPlan((30, 32, 32), 4, 4, "fp32")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("p", [4, 6, 8])
def test_cuda_core_harmonic_compression(orc, prec, tol, p):
    """The CUDA-core M2L on the (p+1)^2 harmonic components (folded multipoles
    in, the c <= 1 locals out, the rest rebuilt before L2L) and on every
    Cartesian component, both against the oracle (FP64 at order 8 keeps the
    Cartesian form: P2M could not stage the folded rows)."""
    shape = (48, 40, 56)
    rho = inputs.lognormal(shape, seed=p).astype(np.float64)
    ref = orc.fmm(rho, 4, p)["phi"]
    dt = torch.float64 if prec == "fp64" else torch.float32
    for harmonic in (True, False):
        plan = fmm.FMMPlan(shape, p, 4, prec, accel=False, harmonic=harmonic)
        phi = plan.solve(torch.from_numpy(rho).cuda().to(dt))
        torch.cuda.synchronize()
        plan.check()
        plan.close()
        err = rel_l2(phi.double().cpu().numpy(), ref)
        print(f"{prec} p={p} harmonic={harmonic}: {err:.2e}")
        assert err <= tol
