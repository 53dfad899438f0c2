"""The algorithmic counts that the benchmark's roofline divides by, checked on
CPU by brute force: the (alpha, beta) pair counts of the M2L (Sec. 2.3,
eq. M2L), Cartesian and harmonic, by enumerating the multi-indices; the
per-level interaction-list totals (Sec. 2.2) against the oracle's own list,
box by box; the level extents against the oracle's hierarchy; and the
near-field pair count (eq. direct) by walking the clipped neighbour boxes."""
import itertools
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SHAPES = [((40, 24, 32), 4), ((24, 20, 44), 4), ((24, 20, 40), 2), ((16, 16, 32), 8)]


def _indices(q_max, harmonic):
    """Multi-indices (a, b, c) with a + b + c <= q_max; harmonic: only c <= 1."""
    return [(a, b, n - a - b) for n in range(q_max + 1) for a in range(n, -1, -1) for b in range(n - a, -1, -1)
            if not (harmonic and n - a - b > 1)]


def test_pair_counts_by_enumeration():
    for p in range(9):
        full = _indices(p, False)
        assert len(full) == math.comb(p + 3, 3)
        assert bench.m2l_pairs(p) == sum(1 for a in full for b in full if sum(a) + sum(b) <= p)
        harm = _indices(p, True)
        assert len(harm) == (p + 1) ** 2
        assert bench.m2l_pairs_harmonic(p) == sum(1 for a in harm for b in harm if sum(a) + sum(b) <= p)
    # p = 6: 84 Cartesian components, 924 pairs; 49 harmonic components, 532 pairs
    assert (bench.m2l_pairs(6), bench.m2l_pairs_harmonic(6)) == (924, 532)


def test_hierarchy_matches_the_oracle(orc):
    for shape, b in SHAPES:
        assert [tuple(e) for e in bench.hierarchy(shape, b)] == [tuple(int(v) for v in r)
                                                                  for r in orc.levels(shape, b)]


def test_interaction_list_totals_match_the_oracle(orc):
    for shape, b in SHAPES:
        lev = orc.levels(shape, b)
        for level in range(2, len(lev)):
            nx, ny, nz = (int(v) for v in lev[level])
            total = sum(orc.ilist_count(shape, b, level, (i, j, k))
                        for k in range(nz) for j in range(ny) for i in range(nx))
            assert bench.il_total((nx, ny, nz)) == total, (shape, b, level)
            assert bench.m2l_flop_level(shape, b, 6, level) == 2 * total * 924
            assert bench.m2l_flop_level(shape, b, 6, level, harmonic=True) == 2 * total * 532
            if level == len(lev) - 1:  # final-stage M2P: every multipole coefficient at every cell
                assert bench.m2p_flop_leaf(shape, b, 6) == 2 * total * 84 * b ** 3
                assert bench.m2p_flop_leaf(shape, b, 6, harmonic=True) == 2 * total * 49 * b ** 3


def test_near_field_pair_count():
    for shape, b in SHAPES:
        nx, ny, nz = bench.hierarchy(shape, b)[-1]
        boxes = 0
        for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
            for dk, dj, di in itertools.product((-1, 0, 1), repeat=3):
                boxes += 0 <= i + di < nx and 0 <= j + dj < ny and 0 <= k + dk < nz
        # every target cell against every cell of each neighbour box: one multiply-add each
        assert bench.algorithmic_counts(shape, b, 4)["near_flop"] == 2 * boxes * b ** 6


def test_batch_roofline_counts():
    """The batch roofline's flops are the per-field counts summed: M2L on the
    harmonic pairs of every level plus every near field; its rate and
    fraction follow from the step time (25.90 ms for the 64-field batch)."""
    from paper_2606_13793_gb300 import inputs
    sizes = inputs.batch_sizes(64, seed=2606)
    want = 0
    for s in sizes:
        lev = bench.hierarchy((s, s, s), 4)
        want += sum(bench.il_total(lev[l]) for l in range(2, len(lev))) * 2 * bench.m2l_pairs_harmonic(6)
        want += bench.algorithmic_counts((s, s, s), 4, 6)["near_flop"]
    assert bench.batch_contraction_flops(sizes, 4, 6) == want
    r = bench.batch_roofline(sizes, 4, 6, "fp32", 25.90, {"sm_max_mhz": 2070.0})
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["flop_per_step"] == want
    assert abs(r["achieved"] - want / 25.90e-3 / 1e12) < 1e-9
    assert abs(r["peak"] - 80.547840) < 1e-6 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert 0.3 < r["frac"] < 0.6  # 36.7 TFLOP/s of 80.5
    r64 = bench.batch_roofline(sizes, 4, 6, "fp64", 100.0, {})
    assert r64["peak"] == 1.25
