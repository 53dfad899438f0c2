"""Pins of the oracle's single operators against closed forms, identities and
the counts the paper prints.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")


def gold(key):
    with open(GOLD) as f:
        return json.load(f)[key]["value"]


# ---------------------------------------------------------------- counts ---

def test_coefficient_counts_match_paper(orc):
    assert orc.ncoef(2) == gold("ncoef_order2")
    assert orc.ncoef(3) == gold("ncoef_order3")
    assert 8 * orc.ncoef(2) == gold("coeffs_per_oct_order2")
    for p in range(0, 11):
        assert orc.ncoef(p) == math.comb(p + 3, 3)


def test_canonical_index_order(orc):
    idx = orc.index(3)
    assert idx.shape == (20, 3)
    assert [tuple(r) for r in idx[:5]] == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0)]
    orders = idx.sum(1)
    assert np.all(np.diff(orders) >= 0)
    assert len({tuple(r) for r in idx}) == 20


def test_interaction_list_geometry(orc):
    # interior target at a level with many boxes: 6^3 - 3^3 = 189 (Sec. 2.2)
    shape, b = (128, 128, 128), 4  # 32^3 leaves, levels 0..5
    L = orc.levels(shape, b).shape[0] - 1
    assert orc.ilist_count(shape, b, L, (15, 16, 17)) == gold("interaction_list_interior")
    assert orc.ilist_count(shape, b, L - 1, (7, 8, 9)) == 189
    # isolated boundary clips the list (corner box)
    corner = orc.ilist_count(shape, b, L, (0, 0, 0))
    assert 0 < corner < 189
    assert corner == 4 ** 3 - 2 ** 3  # parent's neighbours cover [0,4)^3, minus the 2^3 near boxes
    # levels 0 and 1: every box is a neighbour of every other
    assert orc.ilist_count(shape, b, 1, (1, 0, 1)) == 0


def test_level_extents_ceil_halving(orc):
    lv = orc.levels((96, 96, 96), 4)  # 24 -> 12 -> 6 -> 3 -> 2 -> 1
    assert [r[0] for r in lv] == [1, 2, 3, 6, 12, 24]
    lv = orc.levels((64, 32, 16), 4)
    assert tuple(lv[-1]) == (16, 8, 4) and tuple(lv[0]) == (1, 1, 1)


# ------------------------------------------------------------- D tensor ---

def _dt(orc, R, order):
    idx = orc.index(order)
    D = orc.dtensor(R, order)
    return {tuple(r): v for r, v in zip(idx, D)}


def test_dtensor_closed_forms(orc):
    R = np.array([1.3, -0.7, 2.1])
    x, y, z = R
    r = np.linalg.norm(R)
    D = _dt(orc, R, 3)
    # g = -1/r
    exp = {
        (0, 0, 0): -1 / r,
        (1, 0, 0): x / r**3,
        (0, 1, 0): y / r**3,
        (2, 0, 0): (r * r - 3 * x * x) / r**5,
        (1, 1, 0): -3 * x * y / r**5,
        (0, 1, 1): -3 * y * z / r**5,
        (3, 0, 0): 15 * x**3 / r**7 - 9 * x / r**5,
        (2, 1, 0): 15 * x * x * y / r**7 - 3 * y / r**5,
        (1, 1, 1): 15 * x * y * z / r**7,
        (0, 0, 3): 15 * z**3 / r**7 - 9 * z / r**5,
    }
    for k, v in exp.items():
        assert D[k] == pytest.approx(v, rel=1e-13, abs=1e-15), k


def test_dtensor_harmonic_and_parity(orc):
    rng = np.random.default_rng(5)
    for _ in range(5):
        R = rng.uniform(-4, 4, 3)
        R[0] += 6.0
        p = 10
        D = _dt(orc, R, p)
        Dm = _dt(orc, -R, p)
        scale = max(abs(v) for v in D.values())
        for g, v in D.items():
            n = sum(g)
            assert Dm[g] == pytest.approx((-1) ** n * v, rel=1e-12, abs=1e-14 * scale)
            if n <= p - 2:
                lap = D[(g[0] + 2, g[1], g[2])] + D[(g[0], g[1] + 2, g[2])] + D[(g[0], g[1], g[2] + 2)]
                mag = abs(D[(g[0] + 2, g[1], g[2])]) + abs(D[(g[0], g[1] + 2, g[2])]) + abs(D[(g[0], g[1], g[2] + 2)])
                assert abs(lap) <= 1e-11 * mag + 1e-300


def test_dtensor_finite_differences(orc):
    R = np.array([3.2, 1.1, -2.4])
    p = 6
    D = _dt(orc, R, p)
    h = 1e-3
    for q in range(3):
        e = np.zeros(3)
        e[q] = h
        Dp, Dm = _dt(orc, R + e, p - 1), _dt(orc, R - e, p - 1)
        Dp2, Dm2 = _dt(orc, R + 2 * e, p - 1), _dt(orc, R - 2 * e, p - 1)
        for g in Dp:
            fd = (-Dp2[g] + 8 * Dp[g] - 8 * Dm[g] + Dm2[g]) / (12 * h)
            up = list(g)
            up[q] += 1
            assert fd == pytest.approx(D[tuple(up)], rel=1e-7, abs=1e-9 * abs(D[(0, 0, 0)]))


# ---------------------------------------------------------------- P2M -----

def test_p2m_closed_forms(orc):
    p = 4
    idx = orc.index(p)
    # single unit mass: M_alpha = e^alpha
    rho = np.zeros((4, 4, 4))
    rho[1, 3, 0] = 1.0  # cell (x=0, y=3, z=1)
    c = np.array([2.0, 2.0, 2.0])
    M = orc.p2m_region(rho, (0, 0, 0), (4, 4, 4), c, p)
    e = np.array([0.5, 3.5, 1.5]) - c
    for k, a in enumerate(idx):
        assert M[k] == pytest.approx(np.prod(e ** a), rel=1e-15, abs=1e-15)
    # uniform unit block of 4^3 about its centre: cell offsets {+-0.5, +-1.5}
    rho = np.ones((4, 4, 4))
    M = dict(zip(map(tuple, idx), orc.p2m_region(rho, (0, 0, 0), (4, 4, 4), c, p)))
    assert M[(0, 0, 0)] == 64.0
    assert M[(1, 0, 0)] == 0.0 and M[(1, 1, 0)] == 0.0 and M[(3, 0, 0)] == 0.0
    assert M[(2, 0, 0)] == 16 * 2 * (0.25 + 2.25)  # 80
    assert M[(4, 0, 0)] == 16 * 2 * (0.0625 + 5.0625)  # 164
    assert M[(2, 2, 0)] == 4 * 5.0 * 5.0  # 100


def test_p2m_monopole_dipole(orc):
    rng = np.random.default_rng(3)
    rho = rng.uniform(0, 1, (8, 8, 8))
    c = np.array([3.7, 4.2, 5.1])
    M = orc.p2m_region(rho, (0, 0, 0), (8, 8, 8), c, 3)
    z, y, x = np.meshgrid(np.arange(8) + 0.5, np.arange(8) + 0.5, np.arange(8) + 0.5, indexing="ij")
    assert M[0] == pytest.approx(rho.sum(), rel=1e-14)
    assert M[1] == pytest.approx((rho * (x - c[0])).sum(), rel=1e-13)
    assert M[2] == pytest.approx((rho * (y - c[1])).sum(), rel=1e-13)
    assert M[3] == pytest.approx((rho * (z - c[2])).sum(), rel=1e-13)


# ---------------------------------------------------------------- M2M -----

def test_m2m_equals_direct_p2m_about_parent(orc):
    rng = np.random.default_rng(11)
    p = 6
    rho = rng.uniform(0, 2, (8, 8, 8))
    cp = np.array([4.0, 4.0, 4.0])
    Mp_direct = orc.p2m_region(rho, (0, 0, 0), (8, 8, 8), cp, p)
    Mp = np.zeros_like(Mp_direct)
    for cz in range(2):
        for cy in range(2):
            for cx in range(2):
                lo = (4 * cx, 4 * cy, 4 * cz)
                cc = np.array(lo, dtype=float) + 2.0
                Mc = orc.p2m_region(rho, lo, (4, 4, 4), cc, p)
                Mp += orc.m2m(Mc, cc - cp, p)
    np.testing.assert_allclose(Mp, Mp_direct, rtol=1e-12, atol=1e-12 * np.abs(Mp_direct).max())


def test_origin_route_equals_centred_route(orc):
    """Sec. 2.1: origin moments summed then shifted by eq. M2M_general give the
    centred moments (reading Q4)."""
    from paper_2606_13793_gb300 import inputs

    rho = inputs.gaussian_blobs(16, seed=8)
    p = 4
    for level in (1, 2):
        Mo = orc.upward_origin(rho, 4, p, level)
        Mc = orc.fmm(rho, 4, p, export_level=level)["M"]
        np.testing.assert_allclose(Mo, Mc, rtol=1e-9, atol=1e-10 * np.abs(Mc).max())


# ------------------------------------------------------------ L2L / L2P ---

def test_l2l_then_l2p_is_exact(orc):
    rng = np.random.default_rng(21)
    for p in (0, 3, 6):
        Lp = rng.standard_normal(orc.ncoef(p))
        for _ in range(4):
            a = rng.uniform(-2, 2, 3)
            e = rng.uniform(-2, 2, 3)
            Lc = orc.l2l(Lp, a, p)
            assert orc.l2p(Lc, e, p) == pytest.approx(orc.l2p(Lp, a + e, p), rel=1e-12, abs=1e-12)


def test_l2p_closed_form(orc):
    p = 3
    idx = orc.index(p)
    L = np.zeros(len(idx))
    L[idx.tolist().index([2, 0, 1])] = 6.0  # phi = 6 * x^2 z / (2! 1!) = 3 x^2 z
    e = np.array([0.7, -1.1, 0.4])
    assert orc.l2p(L, e, p) == pytest.approx(3 * 0.49 * 0.4, rel=1e-15)


# ---------------------------------------------------------------- M2L -----

def _m2l_point_error(orc, p, src, tgt, cs, ct):
    rho_src = np.array([1.0])
    M = np.array([np.prod((src - cs) ** a) for a in orc.index(p)]) * rho_src[0]
    L = orc.m2l(M, ct - cs, p)
    phi = orc.l2p(L, tgt - ct, p)
    exact = -1.0 / np.linalg.norm(tgt - src)
    return abs(phi - exact) / abs(exact)


def test_m2l_converges_geometrically(orc):
    cs = np.array([0.0, 0.0, 0.0])
    ct = np.array([8.0, 0.0, 0.0])  # two boxes of side 4 apart: nearest list distance
    src = cs + np.array([1.5, -0.5, 0.5])
    tgt = ct + np.array([-0.5, 1.5, -1.5])
    errs = [_m2l_point_error(orc, p, src, tgt, cs, ct) for p in range(0, 13)]
    assert errs[-1] < 1e-4 * errs[0]
    # geometric envelope: the worst error of each block of 4 orders drops >= 5x
    blocks = [max(errs[k:k + 4]) for k in (0, 4, 8)]
    assert blocks[1] < 0.2 * blocks[0] and blocks[2] < 0.2 * blocks[1]


def test_m2l_far_off_axis_is_accurate(orc):
    cs = np.array([0.0, 0.0, 0.0])
    ct = np.array([12.0, -8.0, 4.0])
    src = cs + np.array([-1.5, 0.5, 1.5])
    tgt = ct + np.array([1.5, 1.5, -0.5])
    assert _m2l_point_error(orc, 8, src, tgt, cs, ct) < 2e-6
    assert _m2l_point_error(orc, 12, src, tgt, cs, ct) < 2e-8


# ----------------------------------------------------------------- FD -----

def test_fd_stencils_exact_on_polynomials(orc):
    n = 9
    z, y, x = np.meshgrid(np.arange(n) * 1.0, np.arange(n) * 1.0, np.arange(n) * 1.0, indexing="ij")
    dx = 0.5
    # degree-2 polynomial: every stencil (edge, near-edge, interior) is exact
    phi = 0.3 * x * x - 1.2 * x * y + 0.7 * z * z + 2 * y
    a = orc.fd_accel(phi, dx)
    np.testing.assert_allclose(a[0], -(0.6 * x - 1.2 * y) / dx, atol=1e-12)
    np.testing.assert_allclose(a[1], -(-1.2 * x + 2) / dx, atol=1e-12)
    np.testing.assert_allclose(a[2], -(1.4 * z) / dx, atol=1e-12)
    # degree-4 in x: only the interior 4th-order stencil is exact
    phi = x ** 4 - 2 * x ** 3
    a = orc.fd_accel(phi, 1.0)
    inner = slice(2, n - 2)
    np.testing.assert_allclose(a[0][:, :, inner], -(4 * x ** 3 - 6 * x ** 2)[:, :, inner], atol=1e-9)
    assert np.abs(a[0][:, :, 0] + (4 * x ** 3 - 6 * x ** 2)[:, :, 0]).max() > 1e-3


def test_fd_adjoint_is_transpose(orc):
    rng = np.random.default_rng(4)
    for shape in [(7, 6, 5), (2, 9, 3), (1, 4, 8)]:
        phi = rng.standard_normal(shape)
        g = rng.standard_normal((3,) + shape)
        lhs = np.vdot(g, orc.fd_accel(phi, 0.3))
        rhs = np.vdot(orc.fd_accel_adjoint(g, 0.3), phi)
        assert lhs == pytest.approx(rhs, rel=1e-12)
