"""Batched solves of uneven grids replayed as one CUDA graph (fmm_batch_*).

The graph holds the same kernels as the single solves, with the same plans,
so every field must equal its single solve bit for bit.  One field is also
held to the FP64 oracle at the FP32 tolerance (1e-5 relative L2 on phi).
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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def make(shapes, seed0=40):
    plans = [fmm.FMMPlan(s, 6, 4, "fp32", dx=1.0 / s[0]) for s in shapes]
    rhos = [torch.from_numpy(inputs.plummer(s, seed=seed0 + i)).cuda() for i, s in enumerate(shapes)]
    phis = [p._empty() for p in plans]
    accs = [p._empty((3,)) for p in plans]
    return plans, rhos, phis, accs


def test_batch_equals_single_solves(orc):
    plans, rhos, phis, accs = make(SHAPES)
    batch = fmm.BatchSolver(plans)
    batch.solve(rhos, phis, accs)
    torch.cuda.synchronize()
    for p in plans:
        p.check()
    for p, r, f, a in zip(plans, rhos, phis, accs):
        f1, a1 = p.solve(r, accel=True)
        torch.cuda.synchronize()
        assert torch.equal(f, f1) and torch.equal(a, a1), p.shape
    ref = orc.fmm(rhos[2].double().cpu().numpy(), 4, 6, dx=1.0 / 32)
    assert rel_l2(phis[2].cpu().numpy(), ref["phi"]) <= 1e-5
    assert batch.launches(True) == sum(p.launches(True) for p in plans)
    batch.close()
    for p in plans:
        p.close()


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
        assert torch.equal(f, p.solve(r))
    phis2 = [p._empty() for p in plans]  # new output buffers, no accel: new graph
    batch.solve(rhos, phis2)
    torch.cuda.synchronize()
    for f, f2 in zip(phis, phis2):
        assert torch.equal(f, f2)
    batch.close()
    for p in plans:
        p.close()


def test_batch_on_side_stream_and_bad_args():
    plans, rhos, phis, _ = make(SHAPES[:2])
    batch = fmm.BatchSolver(plans)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        batch.solve(rhos, phis, stream=s)
    s.synchronize()
    for p, r, f in zip(plans, rhos, phis):
        assert torch.equal(f, p.solve(r))
    with pytest.raises(ValueError):
        batch.solve(rhos[:1], phis)
    with pytest.raises(ValueError):
        batch.solve(rhos[::-1], phis)  # shapes do not match the plans
    batch.close()
    for p in plans:
        p.close()
