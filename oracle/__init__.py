"""FP64 CPU oracle for the unigrid FMM Poisson solve (Lee & Teyssier).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path (the CUDA library
under ``paper_2606_13793_gb300/``) never imports, links or executes anything
here, and nothing here imports the product.

The arithmetic lives in ``fmm_oracle.c`` (plain C, FP64, OpenMP over target
boxes); this module only builds it with gcc and marshals numpy arrays.

Parity status of each function (what pins it, see tests/test_oracle_*.py):

* ``dtensor``      pinned: closed forms of orders 0-3, the harmonic identity,
                   parity, finite differences of the order below.
* ``p2m_region``   pinned: closed-form moments of point masses / uniform blocks.
* ``m2m``          pinned: exact against P2M taken directly about the parent.
* ``l2l``, ``l2p`` pinned: re-expansion of a polynomial is exact.
* ``m2l``          pinned: geometric convergence to -m/|r| in the order p;
                   sign of R against the direct sum of an off-centre source.
* ``fmm``          pinned: equals ``direct`` to rounding when every box is a
                   near neighbour (no M2L); converges to ``direct`` with p;
                   closed-form potentials (point mass, uniform sphere,
                   Gaussian); symmetry, linearity and mirror equivariance.
* ``direct``       pinned: closed forms (point mass -m/r, self term -m/dx).
* ``fmm_sample``   pinned: equals ``fmm`` at the sampled cells.
* ``adjoint``      pinned: <u, A v> = <A^T u, v> against ``fmm``.
* ``fd_accel``     pinned: exact on polynomials of the stencils' degree.
* ``m2p_eval``     pinned: its gradient equals the central difference of its
                   potential (an analytic derivative of the same truncated sum).
* ``fmm_accel`` (final_stage "m2p")  pinned: converges to ``direct_accel`` in
                   p; the point-mass closed form; equals the pair-force sum
                   when every box is near; agrees with the stencil gradient of
                   ``fmm_m2p``'s potential in the interior.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_long_p = ctypes.POINTER(ctypes.c_long)


def build(out_path: str | None = None, mutant: int = 0, force: bool = False) -> str:
    """Compile fmm_oracle.c into a shared library with gcc (OpenMP if present).

    ``mutant`` > 0 builds a deliberately broken copy (see ORACLE_MUTANT in the
    C source); only the planted-mistake tests ask for one.
    """
    out = out_path or _LIB_PATH
    if not force and mutant == 0 and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm", f"-DORACLE_MUTANT={mutant}"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    D, I, L, DP, IP, LP = ctypes.c_double, ctypes.c_int, ctypes.c_long, _c_double_p, _c_int_p, _c_long_p
    sig = {
        "oracle_ncoef": (I, [I]),
        "oracle_index": (I, [I, IP]),
        "oracle_dtensor": (I, [DP, I, DP]),
        "oracle_m2m": (I, [DP, DP, I, DP]),
        "oracle_m2l": (I, [DP, DP, I, DP]),
        "oracle_l2l": (I, [DP, DP, I, DP]),
        "oracle_l2p": (D, [DP, DP, I]),
        "oracle_levels": (I, [I, I, I, I, IP]),
        "oracle_ilist_count": (I, [I, I, I, I, I, I, I, I]),
        "oracle_p2m_region": (I, [DP, I, I, I, IP, IP, DP, I, DP]),
        "oracle_upward_origin": (I, [DP, I, I, I, I, I, I, DP]),
        "oracle_fd_accel": (I, [DP, I, I, I, D, DP]),
        "oracle_fd_accel_adjoint": (I, [DP, I, I, I, D, DP]),
        "oracle_max_threads": (I, []),
        "oracle_fmm": (I, [DP, I, I, I, I, I, D, D, DP, DP, DP, DP, I, DP, DP, I]),
        "oracle_direct": (I, [DP, I, I, I, D, D, DP, I]),
        "oracle_fmm_sample": (I, [DP, I, I, I, I, I, D, D, L, LP, DP, DP, I]),
        "oracle_adjoint": (I, [DP, DP, I, I, I, I, I, D, D, DP, I]),
        "oracle_adjoint_analytic": (I, [DP, DP, I, I, I, I, I, D, D, DP, I]),
        "oracle_fmm_accel": (I, [DP, I, I, I, I, I, D, D, DP, I]),
        "oracle_direct_accel": (I, [DP, I, I, I, D, D, DP, I]),
        "oracle_fmm_sample_accel": (I, [DP, I, I, I, I, I, D, D, L, LP, DP, I]),
        "oracle_fmm_m2p": (I, [DP, I, I, I, I, I, D, D, DP, I]),
        "oracle_fmm_orders": (I, [DP, I, I, I, I, I, I, I, I, D, D, DP, I]),
        "oracle_m2p_eval": (I, [DP, I, DP, DP, DP]),
        "oracle_fmm_accel_ex": (I, [DP, I, I, I, I, I, I, D, D, DP, I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load(path: str | None = None):
    """Load (building first if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _dp(a):
    return a.ctypes.data_as(_c_double_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """Thin marshalling layer over one loaded oracle library."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else load()

    # ---- tables -----------------------------------------------------------
    def ncoef(self, p: int) -> int:
        return int(self.lib.oracle_ncoef(p))

    def index(self, p: int) -> np.ndarray:
        """Canonical multi-indices (ncoef, 3): by order, then a desc, b desc."""
        out = np.zeros((self.ncoef(p), 3), dtype=np.int32)
        n = self.lib.oracle_index(p, out.ctypes.data_as(_c_int_p))
        assert n == out.shape[0]
        return out

    def levels(self, shape, b: int) -> np.ndarray:
        """Box counts per level as (L+1, 3) rows of (nx, ny, nz), level 0 first."""
        nx, ny, nz = shape
        buf = np.zeros(3 * 64, dtype=np.int32)
        L = self.lib.oracle_levels(nx, ny, nz, b, buf.ctypes.data_as(_c_int_p))
        if L < 0:
            raise ValueError("bad grid")
        return buf[: 3 * (L + 1)].reshape(L + 1, 3)

    def ilist_count(self, shape, b, level, box) -> int:
        nx, ny, nz = shape
        return int(self.lib.oracle_ilist_count(nx, ny, nz, b, level, *box))

    # ---- single operators -------------------------------------------------
    def dtensor(self, R, order: int) -> np.ndarray:
        R = _f64(R)
        out = np.zeros(self.ncoef(order))
        assert self.lib.oracle_dtensor(_dp(R), order, _dp(out)) == 0
        return out

    def m2m(self, Mc, d, p) -> np.ndarray:
        Mc, d = _f64(Mc), _f64(d)
        out = np.zeros(self.ncoef(p))
        self.lib.oracle_m2m(_dp(Mc), _dp(d), p, _dp(out))
        return out

    def m2l(self, M, R, p) -> np.ndarray:
        M, R = _f64(M), _f64(R)
        out = np.zeros(self.ncoef(p))
        self.lib.oracle_m2l(_dp(M), _dp(R), p, _dp(out))
        return out

    def l2l(self, Lp, a, p) -> np.ndarray:
        Lp, a = _f64(Lp), _f64(a)
        out = np.zeros(self.ncoef(p))
        self.lib.oracle_l2l(_dp(Lp), _dp(a), p, _dp(out))
        return out

    def l2p(self, L, e, p) -> float:
        L, e = _f64(L), _f64(e)
        return float(self.lib.oracle_l2p(_dp(L), _dp(e), p))

    def p2m_region(self, rho, lo, ext, c, p) -> np.ndarray:
        rho = _f64(rho)
        nz, ny, nx = rho.shape
        lo = np.ascontiguousarray(lo, dtype=np.int32)
        ext = np.ascontiguousarray(ext, dtype=np.int32)
        c = _f64(c)
        out = np.zeros(self.ncoef(p))
        self.lib.oracle_p2m_region(_dp(rho), nx, ny, nz, lo.ctypes.data_as(_c_int_p),
                                   ext.ctypes.data_as(_c_int_p), _dp(c), p, _dp(out))
        return out

    def upward_origin(self, rho, b, p, level) -> np.ndarray:
        rho = _f64(rho)
        nz, ny, nx = rho.shape
        lev = self.levels((nx, ny, nz), b)[level]
        out = np.zeros((int(np.prod(lev)), self.ncoef(p)))
        assert self.lib.oracle_upward_origin(_dp(rho), nx, ny, nz, b, p, level, _dp(out)) == 0
        return out

    # ---- whole solves -----------------------------------------------------
    def fmm(self, rho, b: int, p: int, dx: float = 1.0, G: float = 1.0, accel: bool = False,
            split: bool = False, export_level: int = -1, threads: int = 0):
        """FMM solve. Returns dict with phi (and accel[3], phi_far, phi_near, M, L)."""
        rho = _f64(rho)
        nz, ny, nx = rho.shape
        phi = np.zeros_like(rho)
        acc = np.zeros((3,) + rho.shape) if accel else None
        pf = np.zeros_like(rho) if split else None
        pn = np.zeros_like(rho) if split else None
        Mx = Lx = None
        if export_level >= 0:
            lev = self.levels((nx, ny, nz), b)[export_level]
            Mx = np.zeros((int(np.prod(lev)), self.ncoef(p)))
            Lx = np.zeros_like(Mx)
        nul = _c_double_p()
        rc = self.lib.oracle_fmm(_dp(rho), nx, ny, nz, b, p, dx, G, _dp(phi),
                                 _dp(acc) if acc is not None else nul,
                                 _dp(pf) if pf is not None else nul,
                                 _dp(pn) if pn is not None else nul,
                                 export_level,
                                 _dp(Mx) if Mx is not None else nul,
                                 _dp(Lx) if Lx is not None else nul, threads)
        if rc != 0:
            raise ValueError("oracle_fmm rejected its arguments")
        out = {"phi": phi}
        if accel:
            out["accel"] = acc
        if split:
            out["phi_far"], out["phi_near"] = pf, pn
        if export_level >= 0:
            out["M"], out["L"] = Mx, Lx
        return out

    def direct(self, rho, dx: float = 1.0, G: float = 1.0, threads: int = 0) -> np.ndarray:
        rho = _f64(rho)
        nz, ny, nx = rho.shape
        phi = np.zeros_like(rho)
        self.lib.oracle_direct(_dp(rho), nx, ny, nz, dx, G, _dp(phi), threads)
        return phi

    def fmm_accel(self, rho, b: int, p: int, dx: float = 1.0, G: float = 1.0, threads: int = 0,
                  final_stage: str = "m2l") -> np.ndarray:
        """Analytic acceleration [3][nz][ny][nx]: gradient of the leaf local
        expansions plus the near-field pair forces; final_stage "m2p" takes
        the leaf interaction list's M2P gradients at the cell centres instead
        of the leaf M2L (the leaf locals are then the parent's alone)."""
        rho = _f64(rho)
        nz, ny, nx = rho.shape
        acc = np.zeros((3,) + rho.shape)
        if final_stage == "m2l":
            rc = self.lib.oracle_fmm_accel(_dp(rho), nx, ny, nz, b, p, dx, G, _dp(acc), threads)
        else:
            rc = self.lib.oracle_fmm_accel_ex(_dp(rho), nx, ny, nz, b, p, {"m2l": 0, "m2p": 1}[final_stage], dx, G,
                                              _dp(acc), threads)
        if rc != 0:
            raise ValueError("oracle_fmm_accel rejected its arguments")
        return acc

    def m2p_eval(self, M, R, p: int):
        """(phi, grad) of one multipole set M (ncoef(p) coefficients, the
        index order of `index`) evaluated by M2P at the point R."""
        M = np.ascontiguousarray(M, dtype=np.float64)
        R = np.ascontiguousarray(R, dtype=np.float64)
        phi = np.zeros(1)
        g = np.zeros(3)
        if self.lib.oracle_m2p_eval(_dp(M), p, _dp(R), _dp(phi), _dp(g)) != 0:
            raise ValueError("oracle_m2p_eval rejected its arguments")
        return float(phi[0]), g

    def fmm_m2p(self, rho, b: int, p: int, dx: float = 1.0, G: float = 1.0, threads: int = 0) -> np.ndarray:
        """Potential with the paper's final stage: M2P at the cell centres for the
        leaf interaction list (instead of M2L + L2P at the leaf level)."""
        rho = _f64(rho)
        nz, ny, nx = rho.shape
        phi = np.zeros_like(rho)
        if self.lib.oracle_fmm_m2p(_dp(rho), nx, ny, nz, b, p, dx, G, _dp(phi), threads) != 0:
            raise ValueError("oracle_fmm_m2p rejected its arguments")
        return phi

    def fmm_orders(self, rho, b: int, p: int, mult_order: int, local_order: int, final_stage: str = "m2l",
                   dx: float = 1.0, G: float = 1.0, threads: int = 0) -> np.ndarray:
        """Potential with multipoles to order mult_order and locals to order
        local_order inside |alpha| + |beta| <= p; final_stage "m2l" or "m2p"."""
        rho = _f64(rho)
        nz, ny, nx = rho.shape
        phi = np.zeros_like(rho)
        fs = {"m2l": 0, "m2p": 1}[final_stage]
        if self.lib.oracle_fmm_orders(_dp(rho), nx, ny, nz, b, p, mult_order, local_order, fs, dx, G, _dp(phi),
                                      threads) != 0:
            raise ValueError("oracle_fmm_orders rejected its arguments")
        return phi

    def direct_accel(self, rho, dx: float = 1.0, G: float = 1.0, threads: int = 0) -> np.ndarray:
        """O(N^2) pair forces [3][nz][ny][nx]."""
        rho = _f64(rho)
        nz, ny, nx = rho.shape
        acc = np.zeros((3,) + rho.shape)
        self.lib.oracle_direct_accel(_dp(rho), nx, ny, nz, dx, G, _dp(acc), threads)
        return acc

    def fmm_sample_accel(self, rho, b, p, cells, dx=1.0, G=1.0, threads: int = 0) -> np.ndarray:
        """Analytic acceleration at flat cell indices, (n, 3)."""
        rho = _f64(rho)
        nz, ny, nx = rho.shape
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        acc = np.zeros((cells.shape[0], 3))
        if self.lib.oracle_fmm_sample_accel(_dp(rho), nx, ny, nz, b, p, dx, G, cells.shape[0],
                                            cells.ctypes.data_as(_c_long_p), _dp(acc), threads) != 0:
            raise ValueError("oracle_fmm_sample_accel rejected its arguments")
        return acc

    def fmm_sample(self, rho, b, p, cells, dx=1.0, G=1.0, accel=False, threads: int = 0):
        """phi (and accel as (n,3)) at the flat cell indices ``cells``."""
        rho = _f64(rho)
        nz, ny, nx = rho.shape
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        phi = np.zeros(cells.shape[0])
        acc = np.zeros((cells.shape[0], 3)) if accel else None
        rc = self.lib.oracle_fmm_sample(_dp(rho), nx, ny, nz, b, p, dx, G, cells.shape[0],
                                        cells.ctypes.data_as(_c_long_p), _dp(phi),
                                        _dp(acc) if acc is not None else _c_double_p(), threads)
        if rc != 0:
            raise ValueError("oracle_fmm_sample rejected its arguments")
        return (phi, acc) if accel else phi

    def adjoint(self, gphi, gaccel, b, p, dx=1.0, G=1.0, threads: int = 0, analytic: bool = False) -> np.ndarray:
        """grad_rho of <gphi, phi> + <gaccel, accel>: accel by the 5-point
        stencil of phi, or (analytic=True) the force of fmm_accel."""
        gphi = _f64(gphi)
        nz, ny, nx = gphi.shape
        ga = _f64(gaccel) if gaccel is not None else None
        out = np.zeros_like(gphi)
        fn = self.lib.oracle_adjoint_analytic if analytic else self.lib.oracle_adjoint
        rc = fn(_dp(gphi), _dp(ga) if ga is not None else _c_double_p(), nx, ny, nz, b, p, dx, G, _dp(out), threads)
        if rc != 0:
            raise ValueError("oracle_adjoint rejected its arguments")
        return out

    def fd_accel(self, phi, dx=1.0) -> np.ndarray:
        phi = _f64(phi)
        nz, ny, nx = phi.shape
        out = np.zeros((3,) + phi.shape)
        self.lib.oracle_fd_accel(_dp(phi), nx, ny, nz, dx, _dp(out))
        return out

    def fd_accel_adjoint(self, gaccel, dx=1.0) -> np.ndarray:
        ga = _f64(gaccel)
        nz, ny, nx = ga.shape[1:]
        out = np.zeros(ga.shape[1:])
        self.lib.oracle_fd_accel_adjoint(_dp(ga), nx, ny, nz, dx, _dp(out))
        return out

    def max_threads(self) -> int:
        return int(self.lib.oracle_max_threads())
