"""GB300-native unigrid FMM Poisson solver (Lee & Teyssier's cell-based FMM).

This package is a thin Python binding over the C ABI in ``include/fmm.h``
(``libfmm_gb300.so``, built in-tree by ``_build.py``): it marshals pointers,
shapes and the current CUDA stream; every step of the solve runs in the
library's kernels.  PyTorch provides device memory, streams and autograd.

There is no CPU fallback: without the compiled library every call raises.

    plan = FMMPlan((nx, ny, nz), order=6, leaf=4, precision="fp32", dx=1/nx)
    phi, accel = plan.solve(rho, accel=True)       # rho: cuda tensor [nz][ny][nx]
    grad_rho = plan.solve_adjoint(grad_phi, grad_accel)
    phi = FMMSolve.apply(rho, plan)                # differentiable
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfmm_gb300.so")

FMM_OK = 0
STATUS = {0: "FMM_OK", 1: "FMM_ERR_ARG", 2: "FMM_ERR_UNSUPPORTED", 3: "FMM_ERR_ALLOC", 4: "FMM_ERR_CUDA",
          5: "FMM_ERR_NONFINITE", 6: "FMM_ERR_TIMEOUT"}
PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16x3": 3}

# every symbol include/fmm.h declares
EXPORTS = [
    "fmm_default_opts",
    "fmm_plan",
    "fmm_solve",
    "fmm_solve_adjoint",
    "fmm_solve_host",
    "fmm_solve_host_many",
    "fmm_check",
    "fmm_workspace_bytes",
    "fmm_solve_launches",
    "fmm_plan_destroy",
    "fmm_last_error",
    "fmm_debug_level",
    "fmm_plan_leaf_level",
    "fmm_timing_enable",
    "fmm_timing_read",
    "fmm_timing_stage_count",
    "fmm_timing_stage_name",
    "fmm_plan_level_kind",
    "fmm_plan_near_on_tensor_cores",
    "fmm_solve_static",
    "fmm_batch_create",
    "fmm_plan_autotune",
    "fmm_plan_tuning",
    "fmm_plan_set_tuning",
    "fmm_plan_tc_schedule",
    "fmm_plan_set_tc_schedule",
    "fmm_plan_debug_timeout",
    "fmm_batch_solve",
    "fmm_batch_destroy",
    "fmm_batch_launches",
    "fmm_batch_set_fused",
    "fmm_batch_is_fused",
]


class FMMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("dx", ctypes.c_double),
                ("G", ctypes.c_double)]


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("n_fp64_levels", ctypes.c_int), ("accel", ctypes.c_int),
                ("final_stage", ctypes.c_int), ("m2l_cartesian", ctypes.c_int), ("mult_order", ctypes.c_int),
                ("coarse_fp32", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libfmm_gb300.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"{p} is missing: build it with paper_2606_13793_gb300._build.build() "
                              "(there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        lib.fmm_default_opts.argtypes = [ctypes.POINTER(_Opts)]
        lib.fmm_default_opts.restype = None
        lib.fmm_plan.argtypes = [ctypes.POINTER(_Grid), i, i, ctypes.POINTER(_Opts), vp, ctypes.POINTER(vp)]
        lib.fmm_plan.restype = i
        lib.fmm_solve.argtypes = [vp, vp, vp, vp, vp]
        lib.fmm_solve.restype = i
        lib.fmm_solve_adjoint.argtypes = [vp, vp, vp, vp, vp]
        lib.fmm_solve_adjoint.restype = i
        lib.fmm_solve_host.argtypes = [vp, vp, vp, vp, vp]
        lib.fmm_solve_host.restype = i
        lib.fmm_solve_host_many.argtypes = [vp, i, vp, vp, vp, vp]
        lib.fmm_solve_host_many.restype = i
        lib.fmm_check.argtypes = [vp]
        lib.fmm_check.restype = i
        lib.fmm_workspace_bytes.argtypes = [vp]
        lib.fmm_workspace_bytes.restype = sz
        lib.fmm_solve_launches.argtypes = [vp, i]
        lib.fmm_solve_launches.restype = i
        lib.fmm_plan_destroy.argtypes = [vp]
        lib.fmm_plan_destroy.restype = i
        lib.fmm_last_error.argtypes = []
        lib.fmm_last_error.restype = ctypes.c_char_p
        lib.fmm_debug_level.argtypes = [vp, i, i, ctypes.POINTER(ctypes.c_double), sz]
        lib.fmm_debug_level.restype = i
        lib.fmm_plan_leaf_level.argtypes = [vp]
        lib.fmm_plan_leaf_level.restype = i
        lib.fmm_plan_autotune.argtypes = [vp, vp]
        lib.fmm_plan_autotune.restype = i
        lib.fmm_plan_tuning.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i)]
        lib.fmm_plan_tuning.restype = i
        lib.fmm_plan_set_tuning.argtypes = [vp, i, i, i]
        lib.fmm_plan_set_tuning.restype = i
        lib.fmm_plan_tc_schedule.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i)]
        lib.fmm_plan_tc_schedule.restype = i
        lib.fmm_plan_set_tc_schedule.argtypes = [vp, i, i]
        lib.fmm_plan_set_tc_schedule.restype = i
        lib.fmm_plan_debug_timeout.argtypes = [vp]
        lib.fmm_plan_debug_timeout.restype = i
        lib.fmm_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp)]
        lib.fmm_batch_create.restype = i
        lib.fmm_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        lib.fmm_batch_solve.restype = i
        lib.fmm_batch_destroy.argtypes = [vp]
        lib.fmm_batch_destroy.restype = i
        lib.fmm_batch_launches.argtypes = [vp, i]
        lib.fmm_batch_launches.restype = i
        lib.fmm_batch_set_fused.argtypes = [vp, i]
        lib.fmm_batch_set_fused.restype = i
        lib.fmm_batch_is_fused.argtypes = [vp]
        lib.fmm_batch_is_fused.restype = i
        lib.fmm_solve_static.argtypes = [ctypes.POINTER(_Grid), i, i, vp, vp, vp, vp]
        lib.fmm_solve_static.restype = i
        lib.fmm_plan_level_kind.argtypes = [vp, i]
        lib.fmm_plan_level_kind.restype = i
        lib.fmm_plan_near_on_tensor_cores.argtypes = [vp]
        lib.fmm_plan_near_on_tensor_cores.restype = i
        lib.fmm_timing_enable.argtypes = [vp, i]
        lib.fmm_timing_enable.restype = i
        lib.fmm_timing_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), i]
        lib.fmm_timing_read.restype = i
        lib.fmm_timing_stage_count.argtypes = []
        lib.fmm_timing_stage_count.restype = i
        lib.fmm_timing_stage_name.argtypes = [i]
        lib.fmm_timing_stage_name.restype = ctypes.c_char_p
        if path is None:
            _lib = lib
        return lib


def _check(lib, status):
    if status != FMM_OK:
        raise FMMError(status, lib.fmm_last_error().decode(errors="replace"))


def _stream_handle(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class FMMPlan:
    """One solver for a fixed grid shape, order, leaf size and precision.

    A plan runs one call at a time: its solves, adjoints, host solves and
    autotuning share one device workspace, so use a plan from one thread and
    order its calls on one stream (separate plans are independent)."""

    def __init__(self, shape, order: int = 6, leaf: int = 4, precision: str = "fp32", dx: float = 1.0,
                 G: float = 1.0, n_fp64_levels: int = 3, accel=True, final_stage: str = "m2l", harmonic=True,
                 mult_order=None, stream=None, coarse: str = "fp32"):
        import torch

        self.lib = load()
        nx, ny, nz = (int(v) for v in shape)
        self.shape = (nx, ny, nz)
        self.order, self.leaf, self.precision = int(order), int(leaf), precision
        self.dx, self.G = float(dx), float(G)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        if precision not in PRECISION:
            raise ValueError(f"precision must be one of {sorted(PRECISION)}")
        grid = _Grid(nx, ny, nz, self.dx, self.G)
        opts = _Opts()
        self.lib.fmm_default_opts(ctypes.byref(opts))
        opts.precision = PRECISION[precision]
        opts.n_fp64_levels = int(n_fp64_levels)
        # coarse: the precision of those coarse M2L levels in the mixed precisions
        if coarse not in ("fp64", "fp32"):
            raise ValueError("coarse must be 'fp64' or 'fp32'")
        opts.coarse_fp32 = 1 if coarse == "fp32" else 0
        # accel: False (none), True (5-point stencil of phi), "analytic" (gradient
        # of the expansions plus near-field pair forces)
        opts.accel = 2 if accel == "analytic" else (1 if accel else 0)
        # final_stage: "m2l" (M2L + L2P at the leaf level) or "m2p" (the
        # paper's final stage: M2P at the cell centres)
        if final_stage not in ("m2l", "m2p"):
            raise ValueError('final_stage must be "m2l" or "m2p"')
        opts.final_stage = 1 if final_stage == "m2p" else 0
        # harmonic: M2L (and tensor-core M2P) on the (p+1)^2 harmonic
        # components (False: every Cartesian component)
        opts.m2l_cartesian = 0 if harmonic else 1
        # mult_order: multipoles kept to this order (None: the order itself;
        # the paper's split is order 3 with mult_order 2)
        opts.mult_order = -1 if mult_order is None else int(mult_order)
        handle = ctypes.c_void_p()
        _check(self.lib, self.lib.fmm_plan(ctypes.byref(grid), self.order, self.leaf, ctypes.byref(opts),
                                           _stream_handle(stream), ctypes.byref(handle)))
        self._h = handle

    # -- helpers -------------------------------------------------------------
    def _tensor(self, t, name, lead=()):
        import torch

        want = tuple(lead) + (self.shape[2], self.shape[1], self.shape[0])
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype:
            raise TypeError(f"{name} must be {self.dtype}, got {t.dtype}")
        if tuple(t.shape) != want:
            raise ValueError(f"{name} must have shape {want}, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return ctypes.c_void_p(t.data_ptr())

    def _empty(self, lead=()):
        import torch

        return torch.empty(tuple(lead) + (self.shape[2], self.shape[1], self.shape[0]), dtype=self.dtype,
                           device="cuda")

    # -- API -----------------------------------------------------------------
    def solve(self, rho, accel: bool = False, phi_out=None, accel_out=None, stream=None):
        """phi (and accel [3][nz][ny][nx] if asked) of the density rho."""
        r = self._tensor(rho, "rho")
        phi = phi_out if phi_out is not None else self._empty()
        acc = None
        if accel:
            acc = accel_out if accel_out is not None else self._empty((3,))
        _check(self.lib, self.lib.fmm_solve(self._h, r, self._tensor(phi, "phi"),
                                            self._tensor(acc, "accel", (3,)) if acc is not None else None,
                                            _stream_handle(stream)))
        return (phi, acc) if accel else phi

    def solve_adjoint(self, grad_phi=None, grad_accel=None, out=None, stream=None):
        """dLoss/drho from dLoss/dphi and (optionally) dLoss/daccel."""
        gp = self._tensor(grad_phi, "grad_phi") if grad_phi is not None else None
        ga = self._tensor(grad_accel, "grad_accel", (3,)) if grad_accel is not None else None
        g = out if out is not None else self._empty()
        _check(self.lib, self.lib.fmm_solve_adjoint(self._h, gp, ga, self._tensor(g, "grad_rho"),
                                                    _stream_handle(stream)))
        return g

    def solve_host(self, rho_host, phi_host, accel_host=None, stream=None):
        """Host-buffer solve (numpy arrays or pinned CPU tensors); synchronous."""
        def ptr(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                return ctypes.c_void_p(a.data_ptr())
            return ctypes.c_void_p(a.ctypes.data)

        _check(self.lib, self.lib.fmm_solve_host(self._h, ptr(rho_host), ptr(phi_host), ptr(accel_host),
                                                 _stream_handle(stream)))

    def solve_host_many(self, rhos, phis, accels=None, stream=None):
        """Several densities through this plan with host buffers (lists of
        numpy arrays or CPU tensors, pinned for the copies to overlap the
        solves): rhos[i] -> phis[i] (and accels[i] [3][nz][ny][nx]).
        Synchronous."""
        import numpy as np

        n = len(rhos)
        if len(phis) != n or (accels is not None and len(accels) != n):
            raise ValueError("rhos, phis and accels must have the same length")
        esize = 8 if self.precision == "fp64" else 4
        cells = self.shape[0] * self.shape[1] * self.shape[2]

        def ptr(a, name, comps):
            if hasattr(a, "data_ptr"):
                if a.is_cuda or a.element_size() != esize or not a.is_contiguous() or a.numel() != comps * cells:
                    raise ValueError(f"{name} must be a contiguous host buffer of {comps * cells} "
                                     f"{esize}-byte values")
                return a.data_ptr()
            if not isinstance(a, np.ndarray):
                raise TypeError(f"{name} must be a numpy array or a CPU tensor")
            if a.itemsize != esize or not a.flags.c_contiguous or a.size != comps * cells:
                raise ValueError(f"{name} must be a contiguous host buffer of {comps * cells} {esize}-byte values")
            return a.ctypes.data

        arr = ctypes.c_void_p * max(n, 1)
        r = arr(*[ptr(a, "rho", 1) for a in rhos])
        f = arr(*[ptr(a, "phi", 1) for a in phis])
        g = arr(*[ptr(a, "accel", 3) for a in accels]) if accels is not None else None
        _check(self.lib, self.lib.fmm_solve_host_many(self._h, n, r, f, g, _stream_handle(stream)))

    def timing(self, enable: bool = True):
        """Start (clearing) or stop per-stage CUDA-event timing."""
        _check(self.lib, self.lib.fmm_timing_enable(self._h, 1 if enable else 0))

    def timing_read(self):
        """{stage: (total_ms, launches)} since the last enable/read (synchronises)."""
        n = int(self.lib.fmm_timing_stage_count())
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int * n)()
        _check(self.lib, self.lib.fmm_timing_read(self._h, ms, cnt, n))
        return {self.lib.fmm_timing_stage_name(i).decode(): (ms[i], cnt[i]) for i in range(n)}

    def check(self):
        _check(self.lib, self.lib.fmm_check(self._h))

    def debug_level(self, what: str, level: int):
        """One level's multipoles ('M') or locals ('L') as float64 [nbox, ncoef] (canonical order)."""
        import numpy as np

        lv = self.levels()[level]
        nc = (self.order + 1) * (self.order + 2) * (self.order + 3) // 6
        out = np.zeros((int(lv[0] * lv[1] * lv[2]), nc))
        _check(self.lib, self.lib.fmm_debug_level(self._h, 0 if what == "M" else 1, int(level),
                                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size))
        return out

    def levels(self):
        ext = [tuple(v // self.leaf for v in self.shape)]
        while any(e > 1 for e in ext[-1]):
            ext.append(tuple((e + 1) // 2 for e in ext[-1]))
        return ext[::-1]

    @property
    def leaf_level(self) -> int:
        return int(self.lib.fmm_plan_leaf_level(self._h))

    def level_kind(self, level: int) -> str:
        """'none', 'fp32', 'fp64' or 'tensor': how the M2L of that level runs."""
        return {0: "none", 1: "fp32", 2: "fp64", 3: "tensor"}.get(
            int(self.lib.fmm_plan_level_kind(self._h, int(level))), "invalid")

    @property
    def near_on_tensor_cores(self) -> bool:
        return bool(self.lib.fmm_plan_near_on_tensor_cores(self._h))

    @property
    def workspace_bytes(self) -> int:
        return int(self.lib.fmm_workspace_bytes(self._h))

    def autotune(self, stream=None):
        """Time the CUDA-core contraction variants and the two tensor-core
        schedules of each tensor-core contraction; keep the fastest."""
        _check(self.lib, self.lib.fmm_plan_autotune(self._h, _stream_handle(stream)))

    def tuning(self, level: int):
        """(shape, dsplit) of M2L level `level` (-1: near field)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(self.lib, self.lib.fmm_plan_tuning(self._h, int(level), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_tuning(self, level: int, shape: int, dsplit: int):
        _check(self.lib, self.lib.fmm_plan_set_tuning(self._h, int(level), int(shape), int(dsplit)))

    TC_SCHEDULE = {"m2l": 0, "near": 1, "m2p": 2}

    TC_SCHEDULE_NAMES = {0: "span", 1: "prefix", 2: "dedicated"}

    def tc_schedule(self, what: str):
        """("prefix" | "span" | "dedicated" | None, set of available
        schedules) of the tensor-core contraction `what` ("m2l", "near" or
        "m2p"); "dedicated" is the leaf-4 near-field kernel."""
        pre, avail = ctypes.c_int(), ctypes.c_int()
        _check(self.lib, self.lib.fmm_plan_tc_schedule(self._h, self.TC_SCHEDULE[what], ctypes.byref(pre),
                                                        ctypes.byref(avail)))
        names = {n for bit, n in ((1, "span"), (2, "prefix"), (4, "dedicated")) if avail.value & bit}
        return (self.TC_SCHEDULE_NAMES.get(pre.value), names)

    def set_tc_schedule(self, what: str, schedule: str):
        code = {v: k for k, v in self.TC_SCHEDULE_NAMES.items()}.get(schedule)
        if code is None:
            raise ValueError("schedule is 'prefix', 'span' or 'dedicated'")
        _check(self.lib, self.lib.fmm_plan_set_tc_schedule(self._h, self.TC_SCHEDULE[what], code))

    def debug_timeout(self):
        """Test hook: the next solve's first prefix-schedule M2L launch lets
        its bounded waits run out (fmm_plan_debug_timeout)."""
        _check(self.lib, self.lib.fmm_plan_debug_timeout(self._h))

    def launches(self, accel: bool = True) -> int:
        return int(self.lib.fmm_solve_launches(self._h, 1 if accel else 0))

    def close(self):
        """Frees the plan's device memory; later calls on it raise."""
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.fmm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Many independent solves (uneven grids) replayed as one CUDA graph
    (fmm_batch_*): each step kind one launch over every field where the plans
    allow it (fused=True), else the graph of per-plan solves.  The plans must
    outlive the solver."""

    def __init__(self, plans, autotune: bool = True, fused: bool = True):
        self.lib = load()
        self.plans = list(plans)
        if autotune:
            for p in self.plans:
                p.autotune()
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(self.lib, self.lib.fmm_batch_create(arr, len(self.plans), ctypes.byref(h)))
        self._h = h
        _check(self.lib, self.lib.fmm_batch_set_fused(self._h, 1 if fused else 0))

    @property
    def fused(self) -> int:
        """1: the current graph is the fused form, 0: per-plan solves, -1: no solve yet."""
        return int(self.lib.fmm_batch_is_fused(self._h))

    def solve(self, rhos, phis, accels=None, stream=None):
        n = len(self.plans)
        if len(rhos) != n or len(phis) != n or (accels is not None and len(accels) != n):
            raise ValueError("one rho / phi (/ accel) per plan")
        r = (ctypes.c_void_p * n)(*[p._tensor(x, "rho").value for p, x in zip(self.plans, rhos)])
        f = (ctypes.c_void_p * n)(*[p._tensor(x, "phi").value for p, x in zip(self.plans, phis)])
        a = None
        if accels is not None:
            a = (ctypes.c_void_p * n)(*[p._tensor(x, "accel", (3,)).value for p, x in zip(self.plans, accels)])
        _check(self.lib, self.lib.fmm_batch_solve(self._h, r, f, a, _stream_handle(stream)))

    def launches(self, accel: bool = True) -> int:
        return int(self.lib.fmm_batch_launches(self._h, 1 if accel else 0))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.fmm_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_static(rho, order: int = 6, leaf: int = 4, dx: float = 1.0, G: float = 1.0, accel: bool = False,
                 phi_out=None, accel_out=None, stream=None):
    """FP32 solve without a plan and without any device allocation by the
    library (fmm_solve_static): for callers that must not allocate device
    memory while they run.  The workspace is the library's fixed 16 MiB
    static device array (about 64^3 cells at order 6, leaf 4); calls that
    overlap on the GPU share it and race, so keep them on one stream.  The
    output tensors may be passed in so that nothing is allocated here either."""
    import torch

    lib = load()
    if not isinstance(rho, torch.Tensor) or not rho.is_cuda or rho.dtype != torch.float32 or rho.dim() != 3:
        raise TypeError("rho must be a 3-D float32 CUDA tensor [nz][ny][nx]")
    if not rho.is_contiguous():
        raise ValueError("rho must be contiguous")
    if rho.device.index is not None and rho.device.index != torch.cuda.current_device():
        raise ValueError("rho is on %s but the current device is cuda:%d: the library works on the current device"
                         % (rho.device, torch.cuda.current_device()))
    nz, ny, nx = rho.shape

    def _out(t, name, shape):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or t.device != rho.device:
            raise TypeError("%s must be a float32 tensor on %s" % (name, rho.device))
        if tuple(t.shape) != shape:
            raise ValueError("%s must have shape %s, not %s" % (name, shape, tuple(t.shape)))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        return t

    phi = _out(phi_out, "phi_out", (nz, ny, nx)) if phi_out is not None else torch.empty_like(rho)
    acc = None
    if accel:
        acc = (_out(accel_out, "accel_out", (3, nz, ny, nx)) if accel_out is not None else
               torch.empty((3, nz, ny, nx), dtype=torch.float32, device=rho.device))
    grid = _Grid(nx, ny, nz, float(dx), float(G))
    _check(lib, lib.fmm_solve_static(ctypes.byref(grid), int(order), int(leaf), ctypes.c_void_p(rho.data_ptr()),
                                     ctypes.c_void_p(phi.data_ptr()),
                                     ctypes.c_void_p(acc.data_ptr()) if acc is not None else None,
                                     _stream_handle(stream)))
    return (phi, acc) if accel else phi


def _make_autograd():
    import torch

    class FMMSolve(torch.autograd.Function):
        """phi, accel = FMMSolve.apply(rho, plan); backward runs fmm_solve_adjoint.

        The solve is linear in rho, so nothing is saved for the backward pass."""

        @staticmethod
        def forward(ctx, rho, plan):
            ctx.plan = plan
            phi, acc = plan.solve(rho.contiguous(), accel=True)
            return phi, acc

        @staticmethod
        def backward(ctx, grad_phi, grad_accel):
            plan = ctx.plan
            gp = grad_phi.contiguous() if grad_phi is not None else None
            ga = grad_accel.contiguous() if grad_accel is not None else None
            if gp is None and ga is None:
                return None, None
            return plan.solve_adjoint(gp, ga), None

    return FMMSolve


def __getattr__(name):
    if name == "FMMSolve":
        cls = _make_autograd()
        globals()["FMMSolve"] = cls
        return cls
    raise AttributeError(name)
