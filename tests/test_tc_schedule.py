"""The tensor-core schedules, checked on the host without a GPU.

tests/tc_schedule_check.cu compiles the library's own schedule builder
(capi.cu) and checks every M2L (orders 2-8, Cartesian and harmonic, bf16x3
and TF32, multipoles or locals below the order), final-stage M2P and near-
field schedule: TMEM and shared-memory budgets, issuer ownership of the
accumulators, the weight-ring producer's replay (no stall, no overlap), and
the MMAs emulated from the packed, swizzled weight tiles against the direct
contraction with the plan's weight function; then five corruptions planted
in a built schedule must each be caught."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2606_13793_gb300 import _build  # noqa: E402

SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tc_schedule_check.cu")


def test_tensor_core_schedules(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    # the kernels' objects resolve the launch functions capi.cu references
    objs = [os.path.join(_build.BUILD_DIR, os.path.splitext(s)[0] + ".o") for s in _build.SOURCES if s != "capi.cu"]
    _build.build(force=not all(os.path.exists(o) for o in objs))
    exe = str(tmp_path / "tc_schedule_check")
    cmd = [nvcc, *_build.ARCH, "-O1", "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
           "-I", _build.CSRC, SRC, *objs, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 54 and all("uncovered 0" in ln for ln in lines)
    # the check is sharp: five planted corruptions of a built schedule, each caught
    r = subprocess.run([exe, "plant"], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("FAILED") == 5
