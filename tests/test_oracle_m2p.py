"""Pins of the oracle's final-stage M2P (the paper's own final stage, Sec. 4:
the leaf interaction list evaluated by M2P at the cell centres), CPU only,
against the O(N^2) direct sum, the point-mass closed form and the
M2L + L2P solve it replaces (which truncates one more expansion)."""
import numpy as np

from paper_2606_13793_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def test_m2p_equals_direct_when_all_boxes_are_near(orc):
    rho = inputs.gaussian_blobs((8, 8, 8), seed=3)
    d = orc.direct(rho)
    assert np.abs(orc.fmm_m2p(rho, 4, 4) - d).max() <= 1e-13 * np.abs(d).max()


def test_m2p_converges_and_beats_m2l_l2p(orc):
    rho = inputs.gaussian_blobs(32, seed=5)
    d = orc.direct(rho)
    e_m2p = [rel(orc.fmm_m2p(rho, 4, p), d) for p in (2, 4, 6, 8)]
    e_m2l = [rel(orc.fmm(rho, 4, p)["phi"], d) for p in (2, 4, 6, 8)]
    assert all(b < a for a, b in zip(e_m2p, e_m2p[1:])), e_m2p
    assert all(m < l for m, l in zip(e_m2p, e_m2l)), (e_m2p, e_m2l)
    assert e_m2p[3] < 6e-6


def test_m2p_point_mass_closed_form(orc):
    n, src = 32, (9, 20, 13)
    rho = inputs.point_mass(n, src)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - src[0]) ** 2 + (y - src[1]) ** 2 + (z - src[2]) ** 2)
    far = r >= 6
    errs = [rel(orc.fmm_m2p(rho, 4, p)[far], -1.0 / r[far]) for p in (4, 6, 8)]
    assert errs[0] > 3 * errs[1] > 9 * errs[2], errs
    assert errs[2] < 5e-5, errs
