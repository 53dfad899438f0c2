"""Batched solves of uneven grids (fmm_batch_*).

Two forms.  The fused form runs each step kind as one launch over every
field (multi-item kernels reading a per-field argument table); it drops the
neighbour split of the CUDA-core contractions, so its sums may be ordered
differently from a single solve: every field is held to the FP64 oracle
(phi 1e-5, stencil force 1e-4 relative L2 in FP32; 1e-9 in FP64) and to its
single solve (phi 2e-6, force 5e-5).  The per-field form (a CUDA graph of the single
solves) holds the same kernels as the single solves, so it must equal them
bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2606_13793_gb300 as fmm  # noqa: E402
from paper_2606_13793_gb300 import _build, inputs  # noqa: E402

SHAPES = [(64, 64, 64), (96, 96, 96), (32, 48, 40), (128, 128, 128), (64, 64, 64), (96, 64, 32)]


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    assert torch.cuda.is_available()


def rel_l2(a, b):
    a = a.double().cpu().numpy() if hasattr(a, "cpu") else np.asarray(a, np.float64)
    b = b.double().cpu().numpy() if hasattr(b, "cpu") else np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make(shapes, seed0=40, prec="fp32", accel=True):
    plans = [fmm.FMMPlan(s, 6, 4, prec, dx=1.0 / s[0]) for s in shapes]
    dt = np.float64 if prec == "fp64" else np.float32
    rhos = [torch.from_numpy(inputs.plummer(s, seed=seed0 + i).astype(dt)).cuda() for i, s in enumerate(shapes)]
    phis = [p._empty() for p in plans]
    accs = [p._empty((3,)) for p in plans] if accel else None
    return plans, rhos, phis, accs


def close(batch, plans):
    batch.close()
    for p in plans:
        p.close()


def test_fused_batch_every_field_matches_oracle(orc):
    plans, rhos, phis, accs = make(SHAPES)
    batch = fmm.BatchSolver(plans)
    batch.solve(rhos, phis, accs)
    torch.cuda.synchronize()
    assert batch.fused == 1
    for p in plans:
        p.check()
    for s, r, f, a in zip(SHAPES, rhos, phis, accs):
        ref = orc.fmm(r.double().cpu().numpy(), 4, 6, dx=1.0 / s[0], accel=True)
        ep, ea = rel_l2(f, ref["phi"]), rel_l2(a, ref["accel"])
        print(f"{s}: phi {ep:.2e} accel {ea:.2e}")
        assert ep <= 1e-5 and ea <= 1e-4, s
    close(batch, plans)


def test_fused_equals_single_solves_and_per_field_graph_is_exact():
    plans, rhos, phis, accs = make(SHAPES)
    fused = fmm.BatchSolver(plans)
    fused.solve(rhos, phis, accs)
    plain = fmm.BatchSolver(plans, autotune=False, fused=False)
    phis2 = [p._empty() for p in plans]
    accs2 = [p._empty((3,)) for p in plans]
    plain.solve(rhos, phis2, accs2)
    torch.cuda.synchronize()
    assert fused.fused == 1 and plain.fused == 0
    for p, r, f, a, f2, a2 in zip(plans, rhos, phis, accs, phis2, accs2):
        f1, a1 = p.solve(r, accel=True)
        torch.cuda.synchronize()
        assert torch.equal(f2, f1) and torch.equal(a2, a1), p.shape  # the per-field graph: the same kernels
        # two FP32 roundings of the same sums (each about 7e-7 from the
        # oracle); the stencil's differences of phi amplify that in the force
        assert rel_l2(f, f1) <= 2e-6 and rel_l2(a, a1) <= 5e-5, p.shape
    assert plain.launches(True) == sum(p.launches(True) for p in plans)
    fused.close()
    close(plain, plans)


def test_fused_launch_count_of_the_64_field_batch():
    """The 64 uneven fields of the batch benchmark: a few launches per step
    kind, not one set per field."""
    sizes = inputs.batch_sizes(64, seed=2606)
    plans = [fmm.FMMPlan((s, s, s), 6, 4, "fp32", dx=1.0 / s) for s in sizes]
    batch = fmm.BatchSolver(plans, autotune=False)
    n = batch.launches(True)
    per_field = sum(p.launches(True) for p in plans)
    print(f"fused launches {n}, per-field {per_field}")
    assert n <= 30 < per_field
    close(batch, plans)


def test_fused_edge_cases(orc):
    """Fields with the smallest tree (leaf level 2), ragged and flat grids,
    one field alone, no force."""
    shapes = [(16, 16, 16), (16, 24, 16), (40, 24, 8), (8, 64, 12)]
    for sub in (shapes, shapes[1:2]):
        plans, rhos, phis, _ = make(sub, seed0=70, accel=False)
        assert len(sub) == 1 or plans[0].leaf_level == 2
        batch = fmm.BatchSolver(plans, autotune=False)
        batch.solve(rhos, phis)
        torch.cuda.synchronize()
        assert batch.fused == 1
        for s, r, f in zip(sub, rhos, phis):
            ref = orc.fmm(r.double().cpu().numpy(), 4, 6, dx=1.0 / s[0])
            assert rel_l2(f, ref["phi"]) <= 1e-5, s
        close(batch, plans)


def test_fused_fp64_and_forms_that_stay_per_field(orc):
    shapes = [(32, 32, 32), (48, 40, 32)]
    plans, rhos, phis, _ = make(shapes, seed0=80, prec="fp64", accel=False)
    batch = fmm.BatchSolver(plans, autotune=False)
    batch.solve(rhos, phis)
    torch.cuda.synchronize()
    assert batch.fused == 1
    for s, r, f in zip(shapes, rhos, phis):
        ref = orc.fmm(r.cpu().numpy(), 4, 6, dx=1.0 / s[0])
        assert rel_l2(f, ref["phi"]) <= 1e-9, s
    accs = [p._empty((3,)) for p in plans]  # an FP64 force: the per-field graph
    batch.solve(rhos, phis, accs)
    torch.cuda.synchronize()
    assert batch.fused == 0
    close(batch, plans)
    # a tensor-core plan in the batch: the per-field graph
    plans = [fmm.FMMPlan((64, 64, 64), 6, 4, "fp32", dx=1 / 64), fmm.FMMPlan((64, 64, 64), 6, 4, "bf16x3", dx=1 / 64)]
    rhos = [torch.from_numpy(inputs.plummer((64, 64, 64), seed=90)).cuda()] * 2
    phis = [p._empty() for p in plans]
    batch = fmm.BatchSolver(plans, autotune=False)
    batch.solve(rhos, phis)
    torch.cuda.synchronize()
    assert batch.fused == 0
    assert torch.equal(phis[0], plans[0].solve(rhos[0]))
    close(batch, plans)


def test_batch_replay_reads_new_contents_and_new_buffers():
    """Replays read the buffers at launch time; other buffers re-capture."""
    plans, rhos, phis, accs = make(SHAPES[:3])
    batch = fmm.BatchSolver(plans)
    batch.solve(rhos, phis, accs)
    for i, s in enumerate(SHAPES[:3]):  # new contents, same buffers: replay only
        rhos[i].copy_(torch.from_numpy(inputs.plummer(s, seed=90 + i)))
    batch.solve(rhos, phis, accs)
    torch.cuda.synchronize()
    for p, r, f in zip(plans, rhos, phis):
        assert rel_l2(f, p.solve(r)) <= 2e-6
    phis2 = [p._empty() for p in plans]  # new output buffers, no accel: new graph
    batch.solve(rhos, phis2)
    torch.cuda.synchronize()
    for f, f2 in zip(phis, phis2):
        assert torch.equal(f, f2)
    close(batch, plans)


def test_batch_on_side_stream_and_bad_args():
    plans, rhos, phis, _ = make(SHAPES[:2])
    for fused in (True, False):
        batch = fmm.BatchSolver(plans, autotune=False, fused=fused)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            batch.solve(rhos, phis, stream=s)
        s.synchronize()
        for p, r, f in zip(plans, rhos, phis):
            assert rel_l2(f, p.solve(r)) <= 2e-6
        with pytest.raises(ValueError):
            batch.solve(rhos[:1], phis)
        with pytest.raises(ValueError):
            batch.solve(rhos[::-1], phis)  # shapes do not match the plans
        batch.close()
    for p in plans:
        p.close()
