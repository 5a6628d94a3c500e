"""CPU oracle for the compact FMG solver -- TEST INFRASTRUCTURE ONLY.

A plain FP64 C implementation (``cmg_oracle.c``) of the method of
"Multigrid with Linear Storage Complexity" -- compact representation,
Algorithms 1-3, Table 1 precisions, BFP storage -- with every floating-point
operation checked for exactness.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path and never imports it.

Parity pins: see tests/test_oracle_*.py.  Parity unpinned: none of the functions
here; the choice of the 3-D widths b1/b2 and of N is a tuning result, not a
property the paper fixes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cmg_oracle.c")
_HDR = os.path.join(_HERE, "cmg_oracle.h")
_INC = os.path.join(_HERE, "cycle_real.inc")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

U, R, RC, Y = 0, 1, 2, 3
OK, EINVAL, ENOMEM, ERANGE, ECORRUPT = 0, 1, 2, 3, 5


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, OpenMP when available)."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in (_SRC, _HDR, _INC)))
    if not (force or stale):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("Lmax", ctypes.c_int), ("b1", ctypes.c_int),
                ("b2", ctypes.c_int), ("ku", ctypes.c_int), ("kr", ctypes.c_int),
                ("N", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("omega", ctypes.c_double), ("arith", ctypes.c_int), ("coef", ctypes.c_int),
                ("smoother", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            vp, i64, i32, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            sig = {
                "cmgo_encode": (i32, [vp, i64, i32, vp, vp]),
                "cmgo_decode": (i32, [vp, vp, i64, i32, vp]),
                "cmgo_npoints": (i64, [i32, i32]),
                "cmgo_nblocks": (i64, [i32, i32]),
                "cmgo_apply_A": (None, [i32, i32, vp, vp]),
                "cmgo_prolong": (None, [i32, i32, vp, vp]),
                "cmgo_restrict": (None, [i32, i32, vp, vp]),
                "cmgo_create": (vp, [ctypes.POINTER(_Params), i32, vp, i32]),
                "cmgo_destroy": (None, [vp]),
                "cmgo_status": (i32, [vp]),
                "cmgo_inexact": (ctypes.c_longlong, [vp]),
                "cmgo_level": (i32, [vp]),
                "cmgo_rhs_shift": (i32, [vp]),
                "cmgo_width": (i32, [vp, i32, i32]),
                "cmgo_start": (i32, [vp]),
                "cmgo_next_level": (i32, [vp]),
                "cmgo_residual": (i32, [vp]),
                "cmgo_down": (i32, [vp, i32]),
                "cmgo_coarse": (i32, [vp]),
                "cmgo_up": (i32, [vp, i32]),
                "cmgo_vcycle": (i32, [vp]),
                "cmgo_correct": (i32, [vp]),
                "cmgo_ir_iteration": (i32, [vp]),
                "cmgo_fmg": (i32, [vp]),
                "cmgo_get_section": (i32, [vp, i32, i32, vp, vp, vp]),
                "cmgo_set_section": (i32, [vp, i32, i32, i32, vp, vp]),
                "cmgo_decode_solution": (i32, [vp, vp]),
                "cmgo_rhs": (i32, [vp, i32, vp]),
                "cmgo_last_t": (i32, [vp, vp]),
                "cmgo_last_w": (i32, [vp, i32, vp]),
                "cmgo_set_coefficient": (i32, [vp, vp]),
                "cmgo_apply_A_diffusion": (i32, [vp, i32, vp, vp]),
                "cmgo_set_rhs_nodal": (i32, [vp, vp]),
                "cmgo_gradient_k": (i32, [vp, vp, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def npoints(dim: int, level: int) -> int:
    return int(lib().cmgo_npoints(dim, level))


def nblocks(dim: int, level: int) -> int:
    return int(lib().cmgo_nblocks(dim, level))


def level_shape(dim: int, level: int) -> Tuple[int, ...]:
    n = (1 << level) - 1
    return (n, n, n) if dim == 3 else (1, n, n)


# ---------------------------------------------------------------- codec
def encode(x: np.ndarray, W: int) -> Tuple[np.ndarray, np.ndarray, int]:
    x = np.ascontiguousarray(x, dtype=np.float64)
    nb = (x.size + 31) // 32
    words = np.zeros(nb * W, dtype=np.uint32)
    e = np.zeros(nb, dtype=np.int8)
    st = lib().cmgo_encode(_p(x), x.size, W, _p(words), _p(e))
    return words, e, int(st)


def decode(words: np.ndarray, e: np.ndarray, n: int, W: int) -> Tuple[np.ndarray, int]:
    words = np.ascontiguousarray(words, dtype=np.uint32)
    e = np.ascontiguousarray(e, dtype=np.int8)
    x = np.zeros(n, dtype=np.float64)
    st = lib().cmgo_decode(_p(words), _p(e), n, W, _p(x))
    return x, int(st)


# ---------------------------------------------------------------- operators
def apply_A(dim: int, level: int, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    out = np.zeros_like(x)
    lib().cmgo_apply_A(dim, level, _p(x), _p(out))
    return out


def prolong(dim: int, level: int, coarse: np.ndarray) -> np.ndarray:
    coarse = np.ascontiguousarray(coarse, dtype=np.float64).reshape(-1)
    fine = np.zeros(npoints(dim, level), dtype=np.float64)
    lib().cmgo_prolong(dim, level, _p(coarse), _p(fine))
    return fine


def restrict(dim: int, level: int, fine: np.ndarray) -> np.ndarray:
    fine = np.ascontiguousarray(fine, dtype=np.float64).reshape(-1)
    coarse = np.zeros(npoints(dim, level - 1), dtype=np.float64)
    lib().cmgo_restrict(dim, level, _p(fine), _p(coarse))
    return coarse


# ---------------------------------------------------------------- solver
class Oracle:
    """Compact FMG (Algorithm 3) on the CPU, step by step."""

    def __init__(self, dim: int, Lmax: int, tables: np.ndarray, scale_exp: int, *,
                 b1: int, b2: int, N: int, nu1: int, nu2: int, omega: float,
                 ku: int = 2, kr: int = 1, arith: int = 0, coef: int = 0,
                 kfield: Optional[np.ndarray] = None, smoother: int = 0):
        self.dim, self.Lmax = dim, Lmax
        self.params = _Params(dim, Lmax, b1, b2, ku, kr, N, nu1, nu2, omega, arith, coef, smoother)
        self._tables = np.ascontiguousarray(tables, dtype=np.int32)
        assert self._tables.shape[1:] == (dim, (1 << Lmax) - 1)
        self._ctx = lib().cmgo_create(ctypes.byref(self.params), self._tables.shape[0],
                                      _p(self._tables), scale_exp)
        if not self._ctx:
            raise ValueError("cmgo_create rejected the parameters")
        if kfield is not None:
            self.set_coefficient(kfield)

    @classmethod
    def for_problem(cls, prob, **kw) -> "Oracle":
        if getattr(prob, "coef", 0):
            kw.setdefault("coef", 1)
            kw.setdefault("arith", 1)
            kw.setdefault("kfield", prob.kfield())
        return cls(prob.dim, prob.Lmax, prob.tables, prob.scale_exp, **kw)

    def set_coefficient(self, k: np.ndarray):
        """Nodal binary32 coefficient on the finest grid, boundary included."""
        k = np.ascontiguousarray(k, dtype=np.float32)
        n = (1 << self.Lmax) + 1
        assert k.size == n ** self.dim
        self._k = k
        return self._chk(lib().cmgo_set_coefficient(self._ctx, _p(k)), "set_coefficient")

    def set_rhs_nodal(self, g: np.ndarray):
        """Diffusion: nodal right-hand side values at the interior finest nodes."""
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert g.size == ((1 << self.Lmax) - 1) ** self.dim
        self._g = g
        return self._chk(lib().cmgo_set_rhs_nodal(self._ctx, _p(g)), "set_rhs_nodal")

    def gradient_k(self, u: np.ndarray, lam: np.ndarray) -> np.ndarray:
        """dJ/dk at every node (boundary included) for the adjoint state lam."""
        u = np.ascontiguousarray(u, dtype=np.float64).ravel()
        lam = np.ascontiguousarray(lam, dtype=np.float64).ravel()
        N = (1 << self.Lmax) + 1
        out = np.zeros(N ** self.dim)
        self._chk(lib().cmgo_gradient_k(self._ctx, _p(u), _p(lam), _p(out)), "gradient_k")
        return out

    def apply_A_diffusion(self, level: int, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros_like(x)
        self._chk(lib().cmgo_apply_A_diffusion(self._ctx, level, _p(x), _p(out)), "apply_A_diffusion")
        return out

    def close(self):
        if self._ctx:
            lib().cmgo_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- state
    @property
    def status(self) -> int:
        return int(lib().cmgo_status(self._ctx))

    @property
    def inexact(self) -> int:
        return int(lib().cmgo_inexact(self._ctx))

    @property
    def level(self) -> int:
        return int(lib().cmgo_level(self._ctx))

    @property
    def rhs_shift(self) -> int:
        return int(lib().cmgo_rhs_shift(self._ctx))

    def width(self, which: int, level: int) -> int:
        return int(lib().cmgo_width(self._ctx, which, level))

    def _chk(self, st: int, what: str) -> int:
        if st != OK:
            raise RuntimeError("oracle %s failed with status %d" % (what, st))
        return st

    # --- steps
    def start(self):
        return self._chk(lib().cmgo_start(self._ctx), "start")

    def next_level(self):
        return self._chk(lib().cmgo_next_level(self._ctx), "next_level")

    def residual(self):
        return self._chk(lib().cmgo_residual(self._ctx), "residual")

    def down(self, level: int):
        return self._chk(lib().cmgo_down(self._ctx, level), "down")

    def coarse(self):
        return self._chk(lib().cmgo_coarse(self._ctx), "coarse")

    def up(self, level: int):
        return self._chk(lib().cmgo_up(self._ctx, level), "up")

    def vcycle(self):
        return self._chk(lib().cmgo_vcycle(self._ctx), "vcycle")

    def correct(self):
        return self._chk(lib().cmgo_correct(self._ctx), "correct")

    def ir_iteration(self):
        return self._chk(lib().cmgo_ir_iteration(self._ctx), "ir_iteration")

    def fmg(self):
        return self._chk(lib().cmgo_fmg(self._ctx), "fmg")

    # --- data
    def get_section(self, which: int, level: int, words: bool = True):
        nb = nblocks(self.dim, level)
        W = self.width(which, level)
        e = np.zeros(nb, dtype=np.int8)
        vals = np.zeros(npoints(self.dim, level), dtype=np.float64)
        w = np.zeros(nb * max(W, 1), dtype=np.uint32) if (words and 2 <= W <= 32) else None
        st = lib().cmgo_get_section(self._ctx, which, level, _p(w) if w is not None else None,
                                    _p(e), _p(vals))
        self._chk(st, "get_section")
        return w, e, vals.reshape(level_shape(self.dim, level))

    def set_section(self, which: int, level: int, W: int, words: np.ndarray, e: np.ndarray):
        words = np.ascontiguousarray(words, dtype=np.uint32)
        e = np.ascontiguousarray(e, dtype=np.int8)
        return self._chk(lib().cmgo_set_section(self._ctx, which, level, W, _p(words), _p(e)),
                         "set_section")

    def decode_solution(self) -> np.ndarray:
        out = np.zeros(npoints(self.dim, self.level), dtype=np.float64)
        self._chk(lib().cmgo_decode_solution(self._ctx, _p(out)), "decode_solution")
        return out.reshape(level_shape(self.dim, self.level))

    def rhs(self, level: int) -> np.ndarray:
        out = np.zeros(npoints(self.dim, level), dtype=np.float64)
        self._chk(lib().cmgo_rhs(self._ctx, level, _p(out)), "rhs")
        return out.reshape(level_shape(self.dim, level))

    def last_t(self) -> np.ndarray:
        out = np.zeros(npoints(self.dim, self.level), dtype=np.float64)
        self._chk(lib().cmgo_last_t(self._ctx, _p(out)), "last_t")
        return out.reshape(level_shape(self.dim, self.level))

    def last_w(self, level: int) -> np.ndarray:
        out = np.zeros(npoints(self.dim, level), dtype=np.float64)
        self._chk(lib().cmgo_last_w(self._ctx, level, _p(out)), "last_w")
        return out.reshape(level_shape(self.dim, level))
