"""The plan's host-side tables and tensor-core schedules, checked without a GPU.

tests/host_check.cu compiles the library's host code (capi.cu) and:

* checks every tensor-core schedule (M2L at orders 2-8, Cartesian and
  harmonic, bf16x3 and TF32, multipoles or locals below the order; final-stage
  M2P; near field): TMEM and shared-memory budgets, issuer ownership of the
  accumulators, the weight-ring producer's replay (no stall, no overlap), and
  the MMAs emulated from the packed, swizzled weight tiles against the direct
  contraction with the plan's weight function; six corruptions planted in a
  built schedule must each be caught;
* writes the plan's unit-box weight tables (S0 of the path: M2L per neighbour
  parent and child pair, final-stage M2P per cell, near-field kernel), which
  are compared here with the oracle's own operators (Sec. 2.3, eq. M2L; the
  final stage of Sec. 4; eq. direct);
* checks the harmonic compression (fold the multipoles, contract the (p+1)^2
  components, rebuild the locals) against the Cartesian contraction, and that
  harmonic locals stay harmonic under the kernels' L2L shift (which the
  in-place rebuild after L2L relies on), p = 2..8;
* reads the CUDA-core M2L weight tiles (reductions cut to a prefix per tile)
  as the kernels do and checks they give the full contraction;
* runs the kernels' separable M2M / L2L shift helpers on the host, compared
  here with the oracle's M2M (eq. M2M_general) and L2L (eq. L2L);
* replays the fused batch's launch tables (Sec. 2.3's steps over many
  fields, one launch per step kind) built from layout-only plans, with
  planted table corruptions that must each be caught.
"""
import itertools
import math
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2606_13793_gb300 import _build  # noqa: E402

SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "host_check.cu")


@pytest.fixture(scope="module")
def host_check(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    # the kernels' objects resolve the launch functions capi.cu references
    objs = [os.path.join(_build.BUILD_DIR, os.path.splitext(s)[0] + ".o") for s in _build.SOURCES if s != "capi.cu"]
    _build.build(force=not all(os.path.exists(o) for o in objs))
    exe = str(tmp_path_factory.mktemp("host_check") / "host_check")
    cmd = [nvcc, *_build.ARCH, "-O1", "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
           "-I", _build.CSRC, SRC, *objs, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def _run(exe, *args):
    r = subprocess.run([exe, *args], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    return r


def test_tensor_core_schedules(host_check):
    r = _run(host_check)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 54 and all("uncovered 0" in ln for ln in lines)


def test_planted_schedule_corruptions_are_caught(host_check):
    r = _run(host_check, "plant")
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("FAILED") == 6


def test_prefix_schedules(host_check):
    """Every prefix-schedule contraction (M2L p = 2..7 and harmonic p = 8
    cases, final-stage M2P, near field): resources, owner rings, one writer
    per accumulator column, the emulated MMAs against the direct contraction,
    and randomised replays of the barrier protocol (no deadlock, exact parity
    waits)."""
    r = _run(host_check, "prefix")
    assert r.returncode == 0, r.stdout + r.stderr
    built = [ln for ln in r.stdout.splitlines() if "passes" in ln]
    assert len(built) >= 40 and all("uncovered 0" in ln for ln in built)
    assert "prefix schedules built: %d" % len(built) in r.stdout


def test_planted_prefix_mistakes_are_caught(host_check):
    r = _run(host_check, "prefix-plant")
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("FAILED") == 10
    assert "two owners on one ring: 40 of 40" in r.stdout


def test_dedicated_near_field_weights_and_products(host_check):
    """The leaf-4 near-field kernel's weight image (swizzled hi / lo planes)
    decodes to the near-field weights, and its three products reproduce the
    FP64 contraction to the split precision."""
    r = _run(host_check, "near4")
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr


def test_dedicated_near_field_barrier_protocol(host_check):
    """The leaf-4 near-field kernel's rings and accumulator hand-offs replayed
    with random interleavings: every parity wait matches its phase, nothing
    deadlocks, for work lists whose last item has 1 to 4 tiles."""
    r = _run(host_check, "near4-protocol")
    assert r.returncode == 0, r.stdout + r.stderr


def test_m2l_centre_neighbour_block_is_zero(host_check):
    """The CUDA-core M2L kernels skip the centre neighbour's weights: all zero
    for every order, Cartesian and harmonic, while every other neighbour
    block holds interaction-list weights."""
    r = _run(host_check, "centre")
    assert r.returncode == 0, r.stdout + r.stderr


def _cubes(sizes):
    return [str(v) for n in sizes for v in (n, n, n)]


_BATCH_SETS = [
    # the 64-field benchmark batch: sizes {64, 96, 128, 192}^3
    ("fp32", 6, 4, None),
    # uneven, non-cubic grids; grids of one leaf-box row; coarse grids of 12
    # and 6 rows
    ("fp32", 6, 4, ["84", "52", "28", "16", "16", "200", "32", "48", "64", "12", "12", "12", "8", "8", "16",
                    "40", "24", "96"]),
    ("fp32", 4, 2, ["28", "18", "66", "8", "8", "8", "64", "32", "16"]),
    ("fp32", 8, 8, ["64", "64", "64", "128", "64", "32"]),
    ("fp64", 6, 4, ["84", "52", "28", "16", "16", "200", "32", "48", "64", "12", "12", "12", "64", "64", "64"]),
]


@pytest.mark.parametrize("prec,order,leaf,dims", _BATCH_SETS)
def test_fused_batch_tables(host_check, prec, order, leaf, dims):
    """The fused batch's launches and item tables as the library builds them:
    the method's step order per field, every M2L level and near field in one
    contraction launch, block ranges that tile each launch and map back (by
    the kernels' own lookup) to one block of one item, the tile form that
    pads least, z-run tiles covering every row once, the leaf-level L2L in
    the leaf kernel, each item on its own field's buffers."""
    if dims is None:
        from paper_2606_13793_gb300 import inputs
        dims = _cubes(inputs.batch_sizes(64, seed=2606))
    r = _run(host_check, "batch", prec, str(order), str(leaf), *dims)
    assert r.returncode == 0, r.stdout + r.stderr
    assert ": ok" in r.stdout
    if len(dims) == 192:  # the benchmark batch: P2M, 3 M2M, 3 contraction, 4 L2L, leaf, force
        assert " 14 launches" in r.stdout


def test_fused_batch_tables_random_sets(host_check):
    """The same replay over seeded random batches: 1-6 fields of random
    non-cubic extents up to 200 cells, orders 0-8, leaf 2, 4 or 8, FP32 (with
    the stencil force: x extents a multiple of 4) and FP64."""
    import random

    rng = random.Random(2606)
    ran = 0
    for _ in range(40):
        prec = rng.choice(["fp32", "fp64"])
        p, leaf = rng.randint(0, 8), rng.choice([2, 4, 8])
        dims = []
        for _ in range(rng.randint(1, 6)):
            d = [rng.randint(1, 200 // leaf) * leaf for _ in range(3)]
            if prec == "fp32":
                d[0] = (d[0] + 7) // 8 * 8
            dims += [str(v) for v in d]
        r = _run(host_check, "batch", prec, str(p), str(leaf), *dims)
        if "not fusable" in r.stdout:  # a field of a single leaf level or too shallow
            continue
        assert r.returncode == 0 and ": ok" in r.stdout, (prec, p, leaf, dims, r.stdout + r.stderr)
        ran += 1
    assert ran >= 25


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_planted_batch_table_mistakes_are_caught(host_check, prec):
    """Corruptions of a built batch table (a gap between block ranges, a
    launch one block short, a dropped contraction, 6-row items given 8-row
    tiles, a missing z slab, L2L levels swapped, the leaf-level L2L left out,
    the force before the leaf evaluation, two items' inputs swapped) must
    each fail the replay."""
    from paper_2606_13793_gb300 import inputs
    dims = _cubes(inputs.batch_sizes(64, seed=2606)) if prec == "fp32" else _BATCH_SETS[4][3]
    r = _run(host_check, "batch-plant", prec, "6", "4", *dims)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "MISSED" not in r.stdout
    assert r.stdout.count("caught:") >= 7


def test_harmonic_compression_is_exact(host_check):
    r = _run(host_check, "harmonic")
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("harmonic p=") == 7
    # the in-place rebuild after L2L: shifted harmonic locals stay harmonic
    assert r.stdout.count("stay harmonic under L2L") == 7


def test_cuda_core_weight_tiles_hold_every_weight(host_check):
    """The CUDA-core M2L tiles cut each 32-column tile's reduction to the
    prefix its lowest order needs; read as the kernels read them they give
    the full contraction exactly (orders 2-8, both forms, reduced orders)."""
    r = _run(host_check, "cuda-core")
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("cuda-core tiles") == 20


@pytest.fixture(scope="module")
def tables(host_check, tmp_path_factory):
    d = tmp_path_factory.mktemp("tables")
    r = _run(host_check, "tables", str(d))
    assert r.returncode == 0, r.stdout + r.stderr
    return d


def _offsets(d):
    return (d % 3 - 1, (d // 3) % 3 - 1, d // 9 - 1)


def _child_offset(ct, cs, D):
    """c_target - c_source in child boxes: target child ct of the parent at the
    origin, source child cs of the neighbour parent D."""
    return np.array([((ct >> q) & 1) - ((cs >> q) & 1) - 2 * D[q] for q in range(3)], dtype=float)


def _factorials(idx):
    return np.array([math.prod(math.factorial(int(v)) for v in row) for row in idx], dtype=float)


@pytest.mark.parametrize("p,mo,lo", [(3, 3, 3), (4, 4, 4), (4, 3, 4), (4, 4, 3)])
def test_m2l_table_equals_the_oracle_operator(orc, tables, p, mo, lo):
    """Unit-box weights: with child boxes of side 1 the scaled multipoles and
    locals are M and L / beta!, so W[alpha, beta] = L_beta(e_alpha) / beta!
    from the oracle's M2L at R = c_target - c_source, zero for near pairs and
    past the multipole / local limits."""
    nc = orc.ncoef(p)
    K = 8 * nc
    W = np.fromfile(tables / f"m2l_p{p}_mo{mo}_lo{lo}.bin").reshape(27, K, K)
    idx = orc.index(p)
    order = idx.sum(1)
    bfact = _factorials(idx)
    limit = (order[:, None] <= mo) & (order[None, :] <= lo)
    cache = {}
    worst = 0.0
    for d in range(27):
        D = _offsets(d)
        for cs, ct in itertools.product(range(8), range(8)):
            got = W[d, cs::8, ct::8]  # [alpha, beta]
            u = _child_offset(ct, cs, D)
            if np.abs(u).max() < 2:
                assert not got.any()
                continue
            key = tuple(u)
            if key not in cache:
                A = np.stack([orc.m2l(np.eye(nc)[a], u, p) for a in range(nc)])  # [alpha, beta]
                cache[key] = A / bfact[None, :]
            ref = np.where(limit, cache[key], 0.0)
            np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())
            worst = max(worst, float(np.abs(got - ref).max() / np.abs(ref).max()))
    print(f"M2L p={p} mo={mo} lo={lo}: max |plan - oracle| / max |W| = {worst:.1e}")


@pytest.mark.parametrize("p,b", [(3, 2), (4, 4)])
def test_m2p_table_equals_the_oracle_derivatives(orc, tables, p, b):
    """Final-stage M2P (Sec. 4) in leaf-box units: the potential at a cell of
    target child ct from a unit multipole alpha of source child cs is
    (-1)^|alpha| / alpha! D_alpha(R), D = the oracle's derivative tensor of
    -1/r, R = the child offset plus the cell's offset from its box centre."""
    nc = orc.ncoef(p)
    b3 = b ** 3
    W = np.fromfile(tables / f"m2p_p{p}_b{b}.bin").reshape(27, 8 * nc, 8 * b3)
    idx = orc.index(p)
    sign_fact = np.where(idx.sum(1) % 2, -1.0, 1.0) / _factorials(idx)
    for d in range(27):
        D = _offsets(d)
        for cs, ct in itertools.product(range(8), range(8)):
            got = W[d, cs::8, ct * b3:(ct + 1) * b3]  # [alpha, cell]
            u = _child_offset(ct, cs, D)
            if np.abs(u).max() < 2:
                assert not got.any()
                continue
            for cell in range(b3):
                e = np.array([cell % b, (cell // b) % b, cell // (b * b)], dtype=float)
                ref = sign_fact * orc.dtensor(u + (e + 0.5) / b - 0.5, p)
                np.testing.assert_allclose(got[:, cell], ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("p,b", [(3, 2), (4, 4)])
def test_m2p_gradient_table_equals_the_oracle_derivatives(orc, tables, p, b):
    """The final-stage M2P's force columns (App. C, Sec. 4): the derivative of
    the potential at a cell in the target's x_q, in leaf-box units, is
    (-1)^|alpha| / alpha! D_{alpha + e_q}(R), D = the oracle's derivative
    tensor of -1/r to order p + 1; column 0 of each child block is the
    potential table itself."""
    nc = orc.ncoef(p)
    b3 = b ** 3
    W = np.fromfile(tables / f"m2pg_p{p}_b{b}.bin").reshape(27, 8 * nc, 8, 4, b3)
    W1 = np.fromfile(tables / f"m2p_p{p}_b{b}.bin").reshape(27, 8 * nc, 8, b3)
    np.testing.assert_array_equal(W[:, :, :, 0, :], W1)
    idx = orc.index(p)
    idx1 = {tuple(a): i for i, a in enumerate(orc.index(p + 1))}
    sign_fact = np.where(idx.sum(1) % 2, -1.0, 1.0) / _factorials(idx)
    shifted = [np.array([idx1[tuple(a + e)] for a in idx]) for e in np.eye(3, dtype=int)]
    for d in range(27):
        D = _offsets(d)
        for cs, ct in itertools.product(range(8), range(8)):
            u = _child_offset(ct, cs, D)
            got = W[d, cs::8, ct]  # [alpha, comp, cell]
            if np.abs(u).max() < 2:
                assert not got.any()
                continue
            for cell in range(b3):
                e = np.array([cell % b, (cell // b) % b, cell // (b * b)], dtype=float)
                Dt = orc.dtensor(u + (e + 0.5) / b - 0.5, p + 1)
                for q in range(3):
                    ref = sign_fact * Dt[shifted[q]]
                    np.testing.assert_allclose(got[:, 1 + q, cell], ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("b", [2, 4])
def test_near_table_equals_the_kernel(tables, b):
    """Near field (eq. direct), cell units: g(r) = -1/|r| with g(0) = -1, and
    the force columns dg/dx_q = r_q / |r|^3 (zero at r = 0), r = target -
    source over the 27 neighbour boxes."""
    b3 = b ** 3
    W = np.fromfile(tables / f"near_b{b}.bin").reshape(27, b3, 4 * b3)
    cells = np.array([(c % b, (c // b) % b, c // (b * b)) for c in range(b3)], dtype=float)
    for d in range(27):
        r = cells[None, :, :] - cells[:, None, :] - b * np.array(_offsets(d), dtype=float)  # [source, target, 3]
        rn = np.linalg.norm(r, axis=2)
        g = np.where(rn == 0, -1.0, -1.0 / np.where(rn == 0, 1.0, rn))
        np.testing.assert_allclose(W[d, :, :b3], g, rtol=1e-15)
        for q in range(3):
            f = np.where(rn == 0, 0.0, r[:, :, q] / np.where(rn == 0, 1.0, rn) ** 3)
            np.testing.assert_allclose(W[d, :, (q + 1) * b3:(q + 2) * b3], f, rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("p", [3, 6, 8])
def test_kernel_shifts_equal_the_oracle_m2m_and_l2l(orc, tables, p):
    """The kernels' separable shifts along x, y, z in turn (M2M and L2L are
    built from them) against the oracle's eq. M2M_general and eq. L2L: with
    unit box size the scaled multipoles are M and the scaled locals L / beta!,
    so shift_up(M, d) = M2M(M, d) and shift_down(L / beta!, a) = L2L(L, a) /
    beta!.  The first case is a child offset (+-1/2), as the kernels use."""
    nc = orc.ncoef(p)
    bfact = _factorials(orc.index(p))
    up = np.fromfile(tables / f"shift_up_p{p}.bin").reshape(-1, 2 * nc + 3)
    down = np.fromfile(tables / f"shift_down_p{p}.bin").reshape(-1, 2 * nc + 3)
    for row in up:
        M, d, got = row[:nc], row[nc:nc + 3], row[nc + 3:]
        ref = orc.m2m(M, d, p)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
    for row in down:
        Lt, a, got = row[:nc], row[nc:nc + 3], row[nc + 3:]
        ref = orc.l2l(Lt * bfact, a, p) / bfact
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
