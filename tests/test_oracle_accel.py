"""Pins of the oracle's analytic acceleration (the force read off the leaf
local expansions plus the near-field pair forces), CPU only.

Each pin is checked against something other than the oracle's own FMM: the
O(N^2) pair-force sum, the point-mass closed form, Newton's third law of the
pair sum, and the finite-difference gradient of the oracle's potential."""
import numpy as np
import pytest

from paper_2606_13793_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def test_accel_equals_direct_when_all_boxes_are_near(orc):
    """2x2x2 leaf boxes: every box is a near neighbour of every other, so the
    FMM force is the pair-force sum exactly (up to rounding)."""
    rho = inputs.gaussian_blobs((8, 8, 8), seed=3)
    a = orc.fmm_accel(rho, 4, 4)
    d = orc.direct_accel(rho)
    assert np.abs(a - d).max() <= 1e-12 * np.abs(d).max()


def test_accel_converges_to_direct_in_p(orc):
    rho = inputs.gaussian_blobs(32, seed=5)
    d = orc.direct_accel(rho)
    errs = [rel(orc.fmm_accel(rho, 4, p), d) for p in (2, 4, 6, 8)]
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:])), errs
    assert errs[1] < 5e-3 and errs[3] < 3e-4, errs


def test_accel_point_mass_closed_form(orc):
    """One unit mass: away from it the force is -G m r / |r|^3 (physical
    units: cell distance times dx, potential G dx^2 per unit density).  The
    pair-force sum is that closed form exactly; the FMM force, the gradient
    of an expansion truncated at order p, converges to it geometrically in p
    (one order behind the potential: 3.1e-5 for phi at p = 8)."""
    n, dx, G = 32, 0.5, 2.0
    src = (9, 20, 13)
    rho = inputs.point_mass(n, src)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.stack([x - src[0], y - src[1], z - src[2]]).astype(float)
    r2 = (r ** 2).sum(0)
    far = r2 >= 36  # outside the source's near region
    with np.errstate(divide="ignore", invalid="ignore"):
        exact = -G * dx * r / r2 ** 1.5
    d = orc.direct_accel(rho, dx=dx, G=G)
    assert rel(d[:, far], exact[:, far]) < 1e-13
    errs = [rel(orc.fmm_accel(rho, 4, p, dx=dx, G=G)[:, far], exact[:, far]) for p in (4, 6, 8)]
    assert errs[0] > 3 * errs[1] > 9 * errs[2], errs
    assert errs[2] < 2e-3, errs


def test_direct_pair_forces_obey_the_third_law(orc):
    rho = inputs.gaussian_blobs((12, 10, 8), seed=9)
    d = orc.direct_accel(rho)
    total = (d * rho[None]).reshape(3, -1).sum(1)
    assert np.abs(total).max() <= 1e-12 * np.abs(d * rho[None]).sum()


def test_accel_sample_equals_full(orc):
    rho = inputs.lognormal((24, 16, 20), seed=4).astype(np.float64)
    cells = np.array([0, 17, 911, 24 * 16 * 20 - 1, 3000])
    s = orc.fmm_sample_accel(rho, 4, 6, cells)
    f = orc.fmm_accel(rho, 4, 6).reshape(3, -1)[:, cells].T
    assert np.abs(s - f).max() <= 1e-13 * np.abs(f).max()


def test_accel_matches_fd_gradient_of_phi_in_the_interior(orc):
    """The 5-point stencil of the oracle's potential approximates the same
    gradient: they agree to the stencil's truncation error on a smooth field."""
    rho = inputs.gaussian_blobs(32, seed=5, sigma=(4.0, 6.0))
    fd = orc.fmm(rho, 4, 8, accel=True)["accel"]
    an = orc.fmm_accel(rho, 4, 8)
    inner = (slice(None), slice(4, -4), slice(4, -4), slice(4, -4))
    assert rel(fd[inner], an[inner]) < 1e-2


def test_adjoint_of_the_analytic_force_is_its_transpose(orc):
    """<gphi, phi(rho)> + <ga, accel(rho)> = <A^T (gphi, ga), rho> with accel
    the analytic force of fmm_accel: the explicit transpose chain (grad-L2P^T
    into the leaf locals, the shared M2L / L2L / M2M transposes, P2M^T, and
    the near pair forces transposed) against the forward solves."""
    rng = np.random.default_rng(12)
    shape, b, p, dx, G = (16, 24, 20), 4, 4, 0.3, 1.7
    rho = rng.standard_normal(shape[::-1])
    gphi = rng.standard_normal(shape[::-1])
    ga = rng.standard_normal((3,) + shape[::-1])
    phi = orc.fmm(rho, b, p, dx=dx, G=G)["phi"]
    acc = orc.fmm_accel(rho, b, p, dx=dx, G=G)
    lhs = np.vdot(gphi, phi) + np.vdot(ga, acc)
    at = orc.adjoint(gphi, ga, b, p, dx=dx, G=G, analytic=True)
    assert lhs == pytest.approx(np.vdot(at, rho), rel=1e-11)
    # the force part alone, and the potential part equal to the stencil adjoint's
    at_f = orc.adjoint(np.zeros_like(gphi), ga, b, p, dx=dx, G=G, analytic=True)
    assert np.vdot(ga, acc) == pytest.approx(np.vdot(at_f, rho), rel=1e-11)
    np.testing.assert_array_equal(orc.adjoint(gphi, None, b, p, dx=dx, G=G, analytic=True),
                                  orc.adjoint(gphi, None, b, p, dx=dx, G=G))


# ---- the analytic force with the paper's final stage (M2P at the cell centres) ----

def test_m2p_gradient_is_the_derivative_of_m2p(orc):
    """d/dx_q of the M2P sum at a point, against the central difference of the
    same M2P evaluation (step 1e-5 box units): the gradient reads
    D_{alpha + e_q}, a mistake in the index or the sign fails it."""
    rng = np.random.default_rng(3)
    for p in (2, 5, 8):
        M = rng.standard_normal(orc.ncoef(p))
        for R in ([2.3, -1.7, 3.1], [-4.0, 0.4, 2.2], [0.9, 3.3, -2.6]):
            R = np.array(R)
            _, g = orc.m2p_eval(M, R, p)
            h = 1e-5
            fd = np.array([(orc.m2p_eval(M, R + h * e, p)[0] - orc.m2p_eval(M, R - h * e, p)[0]) / (2 * h)
                           for e in np.eye(3)])
            assert np.abs(g - fd).max() <= 1e-6 * max(1.0, np.abs(g).max()), (p, R, g, fd)


def test_m2p_accel_equals_direct_when_all_boxes_are_near(orc):
    rho = inputs.gaussian_blobs((8, 8, 8), seed=3)
    a = orc.fmm_accel(rho, 4, 4, final_stage="m2p")
    d = orc.direct_accel(rho)
    assert np.abs(a - d).max() <= 1e-12 * np.abs(d).max()


def test_m2p_accel_converges_to_direct_in_p(orc):
    rho = inputs.gaussian_blobs(32, seed=5)
    d = orc.direct_accel(rho)
    errs = [rel(orc.fmm_accel(rho, 4, p, final_stage="m2p"), d) for p in (2, 4, 6, 8)]
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:])), errs
    assert errs[1] < 5e-3 and errs[3] < 3e-4, errs


def test_m2p_accel_point_mass_closed_form(orc):
    n, dx, G = 32, 0.5, 2.0
    src = (9, 20, 13)
    rho = inputs.point_mass(n, src)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.stack([x - src[0], y - src[1], z - src[2]]).astype(float)
    r2 = (r ** 2).sum(0)
    far = r2 >= 36
    with np.errstate(divide="ignore", invalid="ignore"):
        exact = -G * dx * r / r2 ** 1.5
    errs = [rel(orc.fmm_accel(rho, 4, p, dx=dx, G=G, final_stage="m2p")[:, far], exact[:, far]) for p in (4, 6, 8)]
    assert errs[0] > 3 * errs[1] > 9 * errs[2], errs
    assert errs[2] < 2e-3, errs


def test_m2p_accel_matches_fd_gradient_of_m2p_phi_in_the_interior(orc):
    rho = inputs.gaussian_blobs(32, seed=5, sigma=(4.0, 6.0))
    phi = orc.fmm_m2p(rho, 4, 8)
    fd = orc.fd_accel(phi)
    an = orc.fmm_accel(rho, 4, 8, final_stage="m2p")
    inner = (slice(None), slice(4, -4), slice(4, -4), slice(4, -4))
    assert rel(fd[inner], an[inner]) < 1e-2
