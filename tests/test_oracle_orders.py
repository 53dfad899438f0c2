"""Separate multipole and local orders (the paper keeps multipoles to order 2
and locals to order 3, Sec. 2.1 and 2.3): oracle_fmm_orders against what the
mathematics fixes.

* Transpose: the kernel of the truncated operator is
  sum_{alpha in A, beta in B} e_s^alpha e_t^beta (-1)^|alpha| D_{alpha+beta}(c_t - c_s) / (alpha! beta!),
  and D_g(-R) = (-1)^|g| D_g(R), so swapping the roles of source and target
  swaps A and B: G(mo, lo)^T = G(lo, mo).  G(2, 3) itself is not symmetric.
* Monopole-only multipoles (mo = 0): the far field depends on each leaf box's
  mass alone, so it is invariant under moving mass inside the boxes.
* Order-0 locals (lo = 0): the far field is constant on every leaf box.
* Uniform density on a power-of-two grid: every box is symmetric under
  inversion through its centre, so odd moments vanish and, for odd p, dropping
  the order-p multipoles changes nothing.
"""
import numpy as np
import pytest

from paper_2606_13793_gb300 import inputs


def _dot(a, b):
    return float(np.sum(a * b))


def test_symmetric_orders_reproduce_the_solves(orc):
    rho = inputs.gaussian_blobs((24, 16, 32), seed=3).astype(np.float64)
    for p in (3, 4):
        assert np.array_equal(orc.fmm_orders(rho, 4, p, p, p), orc.fmm(rho, 4, p)["phi"])
        assert np.array_equal(orc.fmm_orders(rho, 4, p, p, p, "m2p"), orc.fmm_m2p(rho, 4, p))


@pytest.mark.parametrize("p,mo,lo", [(3, 2, 3), (4, 3, 4), (4, 2, 4)])
def test_transpose_swaps_the_orders(orc, p, mo, lo):
    rng = np.random.default_rng(p * 10 + mo)
    u = rng.standard_normal((32, 32, 32))
    v = rng.standard_normal((32, 32, 32))
    a = _dot(u, orc.fmm_orders(v, 4, p, mo, lo))
    b = _dot(orc.fmm_orders(u, 4, p, lo, mo), v)
    c = _dot(orc.fmm_orders(u, 4, p, mo, lo), v)
    scale = np.linalg.norm(u) * np.linalg.norm(orc.fmm_orders(v, 4, p, mo, lo))
    assert abs(a - b) <= 1e-12 * scale
    assert abs(a - c) >= 1e-9 * scale  # the asymmetric split is not self-adjoint


def _far(orc, rho, p, mo, lo):
    return orc.fmm_orders(rho, 4, p, mo, lo) - orc.fmm(rho, 4, p, split=True)["phi_near"]


def test_monopole_only_far_field_ignores_mass_moved_inside_boxes(orc):
    rng = np.random.default_rng(7)
    rho = rng.random((32, 32, 32))
    moved = rho.copy()
    for k in range(8):
        for j in range(8):
            for i in range(8):
                blk = moved[4 * k:4 * k + 4, 4 * j:4 * j + 4, 4 * i:4 * i + 4]
                blk[...] = rng.permutation(blk.ravel()).reshape(4, 4, 4)
    f1, f2 = _far(orc, rho, 4, 0, 4), _far(orc, moved, 4, 0, 4)
    assert np.max(np.abs(f1 - f2)) <= 1e-12 * np.max(np.abs(f1))
    g1, g2 = _far(orc, rho, 4, 1, 4), _far(orc, moved, 4, 1, 4)
    assert np.max(np.abs(g1 - g2)) >= 1e-6 * np.max(np.abs(g1))  # dipoles do see it


def test_order_zero_locals_give_a_constant_far_field_per_box(orc):
    rho = inputs.gaussian_blobs((32, 32, 32), seed=9).astype(np.float64)
    f = _far(orc, rho, 4, 4, 0).reshape(8, 4, 8, 4, 8, 4)
    spread = f.max(axis=(1, 3, 5)) - f.min(axis=(1, 3, 5))
    assert np.max(spread) <= 1e-12 * np.max(np.abs(f))
    g = _far(orc, rho, 4, 4, 1).reshape(8, 4, 8, 4, 8, 4)
    assert np.max(g.max(axis=(1, 3, 5)) - g.min(axis=(1, 3, 5))) >= 1e-6 * np.max(np.abs(g))


def test_uniform_density_has_no_odd_moments(orc):
    rho = np.ones((32, 32, 32))
    full, drop = orc.fmm_orders(rho, 4, 3, 3, 3), orc.fmm_orders(rho, 4, 3, 2, 3)
    assert np.max(np.abs(full - drop)) <= 1e-12 * np.max(np.abs(full))
    blobs = inputs.gaussian_blobs((32, 32, 32), seed=4).astype(np.float64)
    a, b = orc.fmm_orders(blobs, 4, 3, 3, 3), orc.fmm_orders(blobs, 4, 3, 2, 3)
    assert np.max(np.abs(a - b)) >= 1e-8 * np.max(np.abs(a))


def test_papers_configuration_against_the_direct_sum(orc):
    """Multipoles to 2, locals to 3, final-stage M2P, leaf boxes of 2 cells
    (one level below the unigrid, the paper's preferred FMM-1)."""
    rho = inputs.gaussian_blobs((16, 16, 16), seed=5).astype(np.float64)
    ref = orc.direct(rho)
    paper = orc.fmm_orders(rho, 2, 3, 2, 3, "m2p")
    sym = orc.fmm_orders(rho, 2, 3, 3, 3, "m2p")
    e_paper = np.linalg.norm(paper - ref) / np.linalg.norm(ref)
    e_sym = np.linalg.norm(sym - ref) / np.linalg.norm(ref)
    print(f"M<=2, L<=3, M2P, b=2: {e_paper:.2e}; symmetric p=3: {e_sym:.2e}")
    assert e_paper < 1e-2 and e_sym <= e_paper * 1.5
