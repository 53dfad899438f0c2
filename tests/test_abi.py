"""The C-ABI library builds for sm_103a, loads, and exports every symbol
include/fmm.h declares; argument validation answers without a GPU.  CPU only:
no compute call is made."""
import ctypes
import os
import re

import pytest

import paper_2606_13793_gb300 as fmm
from paper_2606_13793_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return fmm.load()


def declared_symbols():
    with open(os.path.join(ROOT, "include", "fmm.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z_0-9]+)\s*\(", text)))


def test_header_declarations_are_exported(lib):
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fmm.EXPORTS) == names


def test_binary_targets_sm103a():
    # the build asks nvcc for sm_103a code only
    assert "arch=compute_103a,code=sm_103a" in _build.ARCH


def _plan(lib, nx=32, ny=32, nz=32, dx=1.0, G=1.0, order=4, leaf=4, prec=1, reserved0=0, **fields):
    grid = fmm._Grid(nx, ny, nz, dx, G)
    opts = fmm._Opts()
    lib.fmm_default_opts(ctypes.byref(opts))
    opts.precision = prec
    opts.reserved[0] = reserved0
    for k, v in fields.items():
        setattr(opts, k, v)
    h = ctypes.c_void_p()
    st = lib.fmm_plan(ctypes.byref(grid), order, leaf, ctypes.byref(opts), None, ctypes.byref(h))
    return st, lib.fmm_last_error().decode()


def test_argument_validation_without_gpu(lib):
    cases = [
        (dict(order=9), "order"),
        (dict(order=-1), "order"),
        (dict(leaf=3), "leaf"),
        (dict(nx=30), "multiple"),
        (dict(ny=0), "positive"),
        (dict(dx=0.0), "dx"),
        (dict(dx=float("nan")), "dx"),
        (dict(prec=7), "precision"),
        (dict(reserved0=1), "reserved"),
        (dict(accel=3), "accel"),
        (dict(final_stage=2), "final_stage"),
        (dict(m2l_cartesian=2), "m2l_cartesian"),
        (dict(mult_order=-2), "mult_order"),
    ]
    for kw, word in cases:
        st, msg = _plan(lib, **kw)
        assert st == 1, (kw, st, msg)  # FMM_ERR_ARG
        assert word in msg, (kw, msg)
    h = ctypes.c_void_p()
    assert lib.fmm_plan(None, 4, 4, None, None, ctypes.byref(h)) == 1
    assert lib.fmm_solve(None, None, None, None, None) == 1
    assert lib.fmm_solve_adjoint(None, None, None, None, None) == 1
    assert lib.fmm_check(None) == 1
    assert lib.fmm_solve_host(None, None, None, None, None) == 1
    assert lib.fmm_solve_host_many(None, 1, None, None, None, None) == 1
    assert "plan is NULL" in lib.fmm_last_error().decode()
    assert lib.fmm_batch_solve(None, None, None, None, None) == 1
    assert lib.fmm_batch_launches(None, 1) == -1
    assert lib.fmm_batch_is_fused(None) == -1
    assert lib.fmm_batch_destroy(None) == 0
    assert lib.fmm_workspace_bytes(None) == 0
    assert lib.fmm_plan_leaf_level(None) == -1
    assert lib.fmm_plan_destroy(None) == 0


def test_binding_rejects_unknown_options(lib):
    # checked in the binding, before any device call
    with pytest.raises(ValueError, match="final_stage"):
        fmm.FMMPlan((8, 8, 8), 2, 4, final_stage="p2p")
    with pytest.raises(ValueError, match="precision"):
        fmm.FMMPlan((8, 8, 8), 2, 4, precision="fp16")


def test_default_options(lib):
    opts = fmm._Opts()
    lib.fmm_default_opts(ctypes.byref(opts))
    assert opts.precision == 1 and opts.n_fp64_levels == 3 and opts.accel == 1
    assert opts.final_stage == 0 and opts.m2l_cartesian == 0 and opts.mult_order == -1
    assert opts.coarse_fp32 == 1 and list(opts.reserved) == [0]


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(ImportError):
        fmm.load(str(tmp_path / "missing.so"))
