"""Pins of the oracle's whole solve: brute force, closed forms, invariants.
CPU only; every case finishes in seconds."""
import math

import numpy as np
import pytest
from scipy.special import erf

from paper_2606_13793_gb300 import inputs


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------ brute force --

@pytest.mark.parametrize("shape,b", [((8, 8, 8), 4), ((4, 4, 4), 2), ((8, 8, 4), 4), ((16, 16, 16), 8), ((4, 2, 4), 2)])
def test_equals_direct_sum_when_all_boxes_are_near(orc, shape, b):
    """n <= 2b per axis: every leaf box is a near neighbour of every other, so
    the FMM is the direct sum (eq. direct) up to rounding."""
    rng = np.random.default_rng(7)
    rho = rng.uniform(0, 1, shape[::-1])
    for p in (0, 4):
        f = orc.fmm(rho, b, p)["phi"]
        d = orc.direct(rho)
        np.testing.assert_allclose(f, d, rtol=1e-13, atol=0)


def test_converges_to_direct_sum_in_p(orc):
    rho = inputs.gaussian_blobs(32, seed=2606)
    d = orc.direct(rho)
    errs = {p: rel_l2(orc.fmm(rho, 4, p)["phi"], d) for p in (2, 4, 6, 8)}
    assert errs[4] < errs[2] and errs[6] < errs[4] and errs[8] < errs[6]
    assert errs[4] < 5e-4 and errs[8] < 2e-5


def test_non_power_of_two_grid_converges(orc):
    rho = inputs.gaussian_blobs((24, 20, 28), seed=9)
    d = orc.direct(rho)
    e4 = rel_l2(orc.fmm(rho, 4, 4)["phi"], d)
    e8 = rel_l2(orc.fmm(rho, 4, 8)["phi"], d)
    assert e8 < e4 < 1e-3


def test_phi_far_plus_near_split(orc):
    rho = inputs.gaussian_blobs(16, seed=4)
    r = orc.fmm(rho, 4, 4, split=True)
    np.testing.assert_allclose(r["phi_far"] + r["phi_near"], r["phi"], rtol=1e-14)
    # the near field is exactly the direct sum over the 27 neighbour boxes
    rho1 = inputs.point_mass(16, (5, 6, 7))
    r1 = orc.fmm(rho1, 4, 4, split=True)
    near = r1["phi_near"]
    assert near[7, 6, 5] == -1.0  # self term g(0) = -1/dx, cell units
    assert near[7, 6, 6] == -1.0  # |r| = 1 = dx
    assert near[7, 6, 7] == pytest.approx(-0.5)
    assert near[7, 6, 12] == 0.0  # leaf box 3 in x is not a neighbour of box 1


# ------------------------------------------------------------ closed forms -

def test_point_mass_closed_form(orc):
    """All mass in one cell: the exact solution of the discrete problem is
    -m/|x - x0| (and -m/dx in the cell itself); the FMM reaches it as p grows."""
    n, cell, m = 32, (9, 20, 14), 2.5
    rho = inputs.point_mass(n, cell, m)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - cell[0]) ** 2.0 + (y - cell[1]) ** 2.0 + (z - cell[2]) ** 2.0)
    exact = np.where(r == 0, -m, -m / np.maximum(r, 1e-300))
    np.testing.assert_allclose(orc.direct(rho), exact, rtol=1e-13)
    e = [rel_l2(orc.fmm(rho, 4, p)["phi"], exact) for p in (2, 4, 8)]
    assert e[2] < e[1] < e[0] and e[2] < 1e-4


def test_point_mass_physical_units(orc):
    rho = inputs.point_mass(16, (8, 8, 8), 1.0)
    dx, G = 1.0 / 16, 3.0
    phi = orc.fmm(rho, 4, 6, dx=dx, G=G)["phi"]
    # mass = rho dx^3; phi = -G mass / (r dx) at r = 4 cells
    expect = -G * dx ** 3 / (4 * dx)
    assert phi[8, 8, 12] == pytest.approx(expect, rel=1e-3)


def test_gaussian_blob_closed_form(orc):
    """A well-resolved Gaussian (sigma = 3 cells): phi = -M erf(r/(sqrt2 s))/r
    up to the discretisation of the mass (small)."""
    n, s, M = 32, 3.0, 1.0
    c = np.array([16.0, 16.0, 16.0])
    z, y, x = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
    rho = M * (2 * np.pi * s * s) ** -1.5 * np.exp(-0.5 * r2 / (s * s))
    r = np.sqrt(r2)
    exact = -rho.sum() * erf(r / (math.sqrt(2) * s)) / r
    phi = orc.fmm(rho, 4, 8)["phi"]
    far = r > 9  # inside, the grid sampling of the blob and g(0) dominate the error
    assert np.abs(phi[far] - exact[far]).max() / np.abs(exact[far]).max() < 1e-3


def test_uniform_sphere_closed_form(orc):
    """The paper's sphere test (Sec. 3): phi = -M/r outside, -M(3R^2-r^2)/(2R^3) inside."""
    n, R0, dens = 32, 7.0, 1.0
    c = (16.0, 16.0, 16.0)
    rho = inputs.uniform_spheres(n, [(c, R0, dens)])
    M = rho.sum()
    z, y, x = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    exact = np.where(r >= R0, -M / np.maximum(r, 1e-9), -M * (3 * R0 * R0 - r * r) / (2 * R0 ** 3))
    phi = orc.fmm(rho, 4, 8)["phi"]
    outside = r > R0 + 2
    assert np.abs(phi[outside] - exact[outside]).max() / np.abs(exact[outside]).max() < 2e-3
    inside = r < R0 - 2
    assert np.abs(phi[inside] - exact[inside]).max() / np.abs(exact[inside]).max() < 3e-2


# ------------------------------------------------------------- invariants --

def test_operator_is_symmetric(orc):
    """With |alpha| + |beta| <= p the FMM operator is symmetric:
    <u, A v> = <A u, v> (reading Q2)."""
    rng = np.random.default_rng(1)
    for shape, b, p in [((32, 32, 32), 4, 4), ((24, 16, 20), 4, 3), ((16, 16, 16), 2, 2)]:
        u = rng.standard_normal(shape[::-1])
        v = rng.standard_normal(shape[::-1])
        lhs = np.vdot(u, orc.fmm(v, b, p)["phi"])
        rhs = np.vdot(orc.fmm(u, b, p)["phi"], v)
        assert lhs == pytest.approx(rhs, rel=1e-11)


def test_adjoint_chain_is_transpose(orc):
    """The explicit transpose chain (oracle.adjoint) satisfies <u, A v> =
    <A^T u, v>, and equals the forward (symmetry), with and without the
    force term."""
    rng = np.random.default_rng(2)
    shape, b, p, dx, G = (16, 16, 24), 4, 4, 0.25, 1.5
    u = rng.standard_normal(shape[::-1])
    v = rng.standard_normal(shape[::-1])
    ga = rng.standard_normal((3,) + shape[::-1])
    fwd = orc.fmm(v, b, p, dx=dx, G=G, accel=True)
    at_u = orc.adjoint(u, None, b, p, dx=dx, G=G)
    assert np.vdot(u, fwd["phi"]) == pytest.approx(np.vdot(at_u, v), rel=1e-11)
    np.testing.assert_allclose(at_u, orc.fmm(u, b, p, dx=dx, G=G)["phi"], rtol=1e-10, atol=1e-12 * np.abs(at_u).max())
    at_full = orc.adjoint(u, ga, b, p, dx=dx, G=G)
    lhs = np.vdot(u, fwd["phi"]) + np.vdot(ga, fwd["accel"])
    assert lhs == pytest.approx(np.vdot(at_full, v), rel=1e-10)


def test_linearity(orc):
    rng = np.random.default_rng(6)
    u = rng.uniform(0, 1, (16, 16, 16))
    v = rng.uniform(0, 1, (16, 16, 16))
    a = orc.fmm(2.5 * u - 0.5 * v, 4, 4)["phi"]
    b = 2.5 * orc.fmm(u, 4, 4)["phi"] - 0.5 * orc.fmm(v, 4, 4)["phi"]
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-12 * np.abs(b).max())


def test_mirror_and_permutation_equivariance(orc):
    rho = inputs.gaussian_blobs(32, seed=12)
    base = orc.fmm(rho, 4, 4)["phi"]
    flipped = orc.fmm(rho[:, :, ::-1].copy(), 4, 4)["phi"]
    np.testing.assert_allclose(flipped, base[:, :, ::-1], rtol=1e-11)
    perm = orc.fmm(np.transpose(rho, (1, 0, 2)).copy(), 4, 4)["phi"]
    np.testing.assert_allclose(perm, np.transpose(base, (1, 0, 2)), rtol=1e-11)


def test_monopole_of_root_is_total_mass(orc):
    rho = inputs.gaussian_blobs((24, 16, 32), seed=3)
    r = orc.fmm(rho, 4, 3, export_level=0)
    assert r["M"][0, 0] == pytest.approx(rho.sum(), rel=1e-13)


def test_sampled_equals_full(orc):
    rho = inputs.gaussian_blobs((32, 24, 16), seed=5)
    full = orc.fmm(rho, 4, 5, dx=0.1, G=2.0, accel=True)
    rng = np.random.default_rng(0)
    cells = rng.integers(0, rho.size, 40)
    cells[:4] = [0, rho.size - 1, 31, 32 * 24 - 1]  # edges
    phi, acc = orc.fmm_sample(rho, 4, 5, cells, dx=0.1, G=2.0, accel=True)
    np.testing.assert_allclose(phi, full["phi"].ravel()[cells], rtol=1e-12)
    for q in range(3):
        np.testing.assert_allclose(acc[:, q], full["accel"][q].ravel()[cells], rtol=1e-9,
                                   atol=1e-11 * np.abs(full["accel"]).max())
