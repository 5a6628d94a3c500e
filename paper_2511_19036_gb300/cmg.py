"""Python binding of the compact FMG library (ctypes; argument marshalling only).

Every computation runs in the CUDA kernels of ``libcmg.so``; this module only
converts arguments.  PyTorch supplies device memory and the CUDA stream.  If the
library has not been built, importing this module raises ImportError.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

from .cmg_config import SolverConfig, config_for  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcmg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libcmg.so is not built; run __graft_entry__.build() (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ERANGE, ECUDA, ECORRUPT, ETIMEOUT, EUNSUPPORTED = range(8)
SEC_U, SEC_R, SEC_RC, SEC_Y = 0, 1, 2, 3
STATUS_NAMES = {0: "CMG_OK", 1: "CMG_EINVAL", 2: "CMG_ENOMEM", 3: "CMG_ERANGE", 4: "CMG_ECUDA",
                5: "CMG_ECORRUPT", 6: "CMG_ETIMEOUT", 7: "CMG_EUNSUPPORTED"}


class CmgError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        super().__init__("%s failed: %s%s" % (where, STATUS_NAMES.get(status, str(status)),
                                              (" (" + detail + ")") if detail else ""))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("L_max", ctypes.c_int), ("b1", ctypes.c_int),
                ("b2", ctypes.c_int), ("k_u", ctypes.c_int), ("k_r", ctypes.c_int),
                ("N_ir", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("omega_num", ctypes.c_int), ("omega_log2den", ctypes.c_int),
                ("arith", ctypes.c_int), ("coef", ctypes.c_int), ("smoother", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("solve_ms", ctypes.c_double), ("dofs", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("alg_bytes", ctypes.c_double),
                ("persistent_bits", ctypes.c_double), ("temp_bytes", ctypes.c_double),
                ("sweep_ms_total", ctypes.c_double), ("sweep_launches", ctypes.c_int64),
                ("sweep_alg_bytes", ctypes.c_double), ("resid_ms_total", ctypes.c_double),
                ("resid_launches", ctypes.c_int64), ("resid_alg_bytes", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp, _i64, _i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
class Storage(ctypes.Structure):
    _fields_ = [("dofs", ctypes.c_double), ("cmg_vector_bits", ctypes.c_double),
                ("cmg_fmg_bits", ctypes.c_double), ("bfpmg_vector_bits", ctypes.c_double),
                ("bfpmg_fmg_bits", ctypes.c_double), ("vector_saving", ctypes.c_double),
                ("fmg_saving", ctypes.c_double)]


_SIGS = {
    "cmg_encode": (_i32, [_vp, _i64, _i32, _vp, _vp, _vp]),
    "cmg_decode": (_i32, [_vp, _vp, _i64, _i32, _vp, _vp]),
    "cmg_params_check": (_i32, [ctypes.POINTER(Params)]),
    "cmg_create": (_i32, [ctypes.POINTER(Params), _vp, ctypes.POINTER(_vp)]),
    "cmg_destroy": (None, [_vp]),
    "cmg_last_error": (ctypes.c_char_p, [_vp]),
    "cmg_set_timing": (_i32, [_vp, _i32]),
    "cmg_set_fast_kernels": (_i32, [_vp, _i32]),
    "cmg_set_two_level": (_i32, [_vp, _i32]),
    "cmg_set_graphs": (_i32, [_vp, _i32]),
    "cmg_graph_stats": (_i32, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "cmg_fast_stats": (_i32, [_vp, _i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "cmg_set_rhs_separable": (_i32, [_vp, _i32, _vp, _i32]),
    "cmg_fmg_solve": (_i32, [_vp, ctypes.POINTER(Report)]),
    "cmg_start": (_i32, [_vp]),
    "cmg_prolongate": (_i32, [_vp]),
    "cmg_residual": (_i32, [_vp]),
    "cmg_down": (_i32, [_vp, _i32]),
    "cmg_coarse": (_i32, [_vp]),
    "cmg_up": (_i32, [_vp, _i32]),
    "cmg_smooth": (_i32, [_vp, _i32, _i32, _i32]),
    "cmg_restrict": (_i32, [_vp, _i32]),
    "cmg_correct": (_i32, [_vp]),
    "cmg_vcycle": (_i32, [_vp]),
    "cmg_ir_iteration": (_i32, [_vp]),
    "cmg_level": (_i32, [_vp]),
    "cmg_sync": (_i32, [_vp]),
    "cmg_section_blocks": (_i64, [_i32, _i32]),
    "cmg_section_width": (_i32, [_vp, _i32, _i32]),
    "cmg_get_section": (_i32, [_vp, _i32, _i32, _vp, _vp]),
    "cmg_set_section": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp]),
    "cmg_decode_solution": (_i32, [_vp, _i64, _i64, _vp]),
    "cmg_state_save": (_i32, [_vp, _vp, ctypes.POINTER(ctypes.c_size_t)]),
    "cmg_state_load": (_i32, [_vp, _vp, ctypes.c_size_t]),
    "cmg_set_coefficient": (_i32, [_vp, _vp, _i64]),
    "cmg_set_rhs_nodal": (_i32, [_vp, _vp, _i64, _i32]),
    "cmg_gradient": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "cmg_storage_model": (_i32, [_i32, _i32, _i32, _i32, _i32, _i32, ctypes.POINTER(Storage)]),
    "cmg_kernel_stats": (_i32, [_vp, _i32, _i32, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
    "cmg_decode_compact_scratch_bytes": (ctypes.c_size_t, [_i32, _i32]),
    "cmg_decode_compact": (_i32, [_i32, _i32, _vp, _vp, _vp, _i64, _i64, _vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def lib() -> ctypes.CDLL:
    return _lib


def storage_model(dim: int, L: int, k_u: int, k_r: int, b1: int, b2: int) -> dict:
    """Sec. 6.1.4 mantissa bits of CMG and BFPMG storage (see cmg_storage_model)."""
    out = Storage()
    st = _lib.cmg_storage_model(dim, L, k_u, k_r, b1, b2, ctypes.byref(out))
    if st != OK:
        raise CmgError(st, "cmg_storage_model", "invalid arguments")
    return {name: getattr(out, name) for name, _ in Storage._fields_}


def exported_symbols():
    return list(_SIGS)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    return t.data_ptr()


# ---------------------------------------------------------------- codec
def encode(x, W: int, stream=None):
    """BFP-encode a CUDA float64 tensor (flattened) into (words uint32-as-int32, exps int8)."""
    import torch
    assert x.is_cuda and x.dtype == torch.float64
    x = x.contiguous().reshape(-1)
    n = x.numel()
    nb = (n + 31) // 32
    words = torch.empty(nb * W, dtype=torch.int32, device=x.device)
    exps = torch.empty(nb, dtype=torch.int8, device=x.device)
    st = _lib.cmg_encode(_ptr(x), n, W, _ptr(words), _ptr(exps), _stream_handle(stream))
    if st != OK:
        raise CmgError(st, "cmg_encode")
    return words, exps


def decode(words, exps, n: int, W: int, stream=None):
    import torch
    x = torch.empty(n, dtype=torch.float64, device=words.device)
    st = _lib.cmg_decode(_ptr(words), _ptr(exps), n, W, _ptr(x), _stream_handle(stream))
    if st != OK:
        raise CmgError(st, "cmg_decode")
    return x


def encode_raw(x_ptr: int, n: int, W: int, words_ptr: int, exps_ptr: int, stream: int) -> int:
    return int(_lib.cmg_encode(x_ptr, n, W, words_ptr, exps_ptr, stream))


def decode_raw(words_ptr: int, exps_ptr: int, n: int, W: int, x_ptr: int, stream: int) -> int:
    return int(_lib.cmg_decode(words_ptr, exps_ptr, n, W, x_ptr, stream))


# ---------------------------------------------------------------- solver
def to_params(cfg: SolverConfig) -> Params:
    return Params(cfg.dim, cfg.L_max, cfg.b1, cfg.b2, cfg.k_u, cfg.k_r, cfg.N_ir,
                  cfg.nu1, cfg.nu2, cfg.omega_num, cfg.omega_log2den, cfg.arith, cfg.coef, cfg.smoother)


def params_check(cfg: SolverConfig) -> int:
    p = to_params(cfg)
    return int(_lib.cmg_params_check(ctypes.byref(p)))


class Solver:
    """Compact FMG context on the current CUDA device."""

    def __init__(self, cfg: SolverConfig, stream=None, timing: bool = False, fast: bool = True,
                 two_level=None, graphs: bool = True):
        self.cfg = cfg
        self._p = to_params(cfg)
        self._stream = _stream_handle(stream)
        h = _vp()
        st = _lib.cmg_create(ctypes.byref(self._p), self._stream, ctypes.byref(h))
        if st != OK:
            raise CmgError(st, "cmg_create")
        self._h = h
        if timing:
            self.set_timing(timing)
        if not fast:
            _lib.cmg_set_fast_kernels(self._h, 0)
        if two_level is not None:
            self.set_two_level(two_level)
        if not graphs:
            self.set_graphs(False)

    def set_timing(self, timing):
        """Per-launch CUDA events: False (none), True (every launch) or "top"
        (launches on level L_max only, see cmg_set_timing)."""
        mode = 2 if timing == "top" else (1 if timing else 0)
        self._chk(_lib.cmg_set_timing(self._h, mode), "cmg_set_timing")

    def set_graphs(self, enable: bool):
        """Solve through a CUDA graph of the whole solve (see cmg_set_graphs)."""
        self._chk(_lib.cmg_set_graphs(self._h, 1 if enable else 0), "cmg_set_graphs")

    def graph_stats(self) -> dict:
        """Graphs captured and solves run as a graph launch since the context was made."""
        c, n = ctypes.c_int64(), ctypes.c_int64()
        self._chk(_lib.cmg_graph_stats(self._h, ctypes.byref(c), ctypes.byref(n)), "cmg_graph_stats")
        return {"captures": c.value, "graph_solves": n.value}

    def set_two_level(self, enable: bool):
        """Finest level's coarse sources formed on the fly (see cmg_set_two_level)."""
        self._chk(_lib.cmg_set_two_level(self._h, 1 if enable else 0), "cmg_set_two_level")

    def close(self):
        if getattr(self, "_h", None):
            _lib.cmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st: int, where: str):
        if st != OK:
            raise CmgError(st, where, _lib.cmg_last_error(self._h).decode(errors="replace"))

    @property
    def level(self) -> int:
        return int(_lib.cmg_level(self._h))

    def set_rhs(self, tables: np.ndarray, scale_exp: int):
        t = np.ascontiguousarray(tables, dtype=np.int32)
        self._chk(_lib.cmg_set_rhs_separable(self._h, t.shape[0], t.ctypes.data, scale_exp),
                  "cmg_set_rhs_separable")

    def fmg_solve(self) -> dict:
        rep = Report()
        self._chk(_lib.cmg_fmg_solve(self._h, ctypes.byref(rep)), "cmg_fmg_solve")
        return rep.as_dict()

    KINDS = ("residual", "sweep", "restrict", "acc_encode", "coarse", "repack", "other")

    def kernel_stats(self) -> dict:
        """Per kernel kind and level class ('top' = L_max): ms, launches, bytes."""
        out = {}
        for kind, name in enumerate(self.KINDS):
            for top in (1, 0):
                ms, n, by = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
                self._chk(_lib.cmg_kernel_stats(self._h, kind, top, ctypes.byref(ms), ctypes.byref(n),
                                                ctypes.byref(by)), "cmg_kernel_stats")
                out["%s_%s" % (name, "top" if top else "lower")] = {
                    "ms": ms.value, "launches": n.value, "bytes": by.value}
        return out

    def fast_stats(self) -> dict:
        """CTAs of the specialised kernels since the solve started, and how many left
        their tile to the generic kernel (all levels and the finest level)."""
        out = {}
        for top, name in ((0, "all"), (1, "top")):
            n, fb = ctypes.c_int64(), ctypes.c_int64()
            self._chk(_lib.cmg_fast_stats(self._h, top, ctypes.byref(n), ctypes.byref(fb)), "cmg_fast_stats")
            out[name] = {"ctas": n.value, "fallback_ctas": fb.value}
        return out

    def set_coefficient(self, k):
        """Diffusion: the nodal binary32 coefficient (CUDA tensor, boundary included,
        (2^L_max + 1)^dim values).  The solver borrows it; it is kept referenced here."""
        import torch
        assert k.is_cuda and k.dtype == torch.float32 and k.is_contiguous()
        self._kfield = k
        self._chk(_lib.cmg_set_coefficient(self._h, k.data_ptr(), k.numel()), "cmg_set_coefficient")

    def set_rhs_nodal(self, g, scale_log2: int = 0):
        """Diffusion: nodal right-hand side 2^scale_log2 g (CUDA float64 tensor, interior
        finest nodes); borrowed, kept referenced here."""
        import torch
        assert g.is_cuda and g.dtype == torch.float64 and g.is_contiguous()
        self._grhs = g
        self._chk(_lib.cmg_set_rhs_nodal(self._h, g.data_ptr(), g.numel(), int(scale_log2)),
                  "cmg_set_rhs_nodal")

    def gradient(self, u, lam, want_dg: bool = True):
        """Adjoint gradients (dJ/dk on every node, dJ/dg on the interior) from the
        state u and the adjoint state lam (CUDA float64, interior)."""
        import torch
        N = (1 << self.cfg.L_max) + 1
        dk = torch.empty(N ** self.cfg.dim, dtype=torch.float64, device=u.device)
        dg = torch.empty_like(lam) if want_dg else None
        self._chk(_lib.cmg_gradient(self._h, u.contiguous().data_ptr(), lam.contiguous().data_ptr(),
                                    dk.data_ptr(), dg.data_ptr() if dg is not None else None), "cmg_gradient")
        return dk, dg

    def start(self):
        self._chk(_lib.cmg_start(self._h), "cmg_start")

    def prolongate(self):
        self._chk(_lib.cmg_prolongate(self._h), "cmg_prolongate")

    def residual(self):
        self._chk(_lib.cmg_residual(self._h), "cmg_residual")

    def down(self, level: int):
        self._chk(_lib.cmg_down(self._h, level), "cmg_down")

    def coarse(self):
        self._chk(_lib.cmg_coarse(self._h), "cmg_coarse")

    def up(self, level: int):
        self._chk(_lib.cmg_up(self._h, level), "cmg_up")

    def smooth(self, level: int, sweeps: int, with_z: bool):
        self._chk(_lib.cmg_smooth(self._h, level, sweeps, int(bool(with_z))), "cmg_smooth")

    def restrict(self, level: int):
        self._chk(_lib.cmg_restrict(self._h, level), "cmg_restrict")

    def correct(self):
        self._chk(_lib.cmg_correct(self._h), "cmg_correct")

    def vcycle(self):
        self._chk(_lib.cmg_vcycle(self._h), "cmg_vcycle")

    def ir_iteration(self):
        self._chk(_lib.cmg_ir_iteration(self._h), "cmg_ir_iteration")

    def sync(self):
        self._chk(_lib.cmg_sync(self._h), "cmg_sync")

    def width(self, which: int, level: int) -> int:
        return int(_lib.cmg_section_width(self._h, which, level))

    def get_section(self, which: int, level: int) -> Tuple[np.ndarray, np.ndarray]:
        nb = int(_lib.cmg_section_blocks(self.cfg.dim, level))
        W = self.width(which, level)
        words = np.zeros(nb * W, dtype=np.uint32)
        exps = np.zeros(nb, dtype=np.int8)
        self._chk(_lib.cmg_get_section(self._h, which, level, words.ctypes.data, exps.ctypes.data),
                  "cmg_get_section")
        return words, exps

    def set_section(self, which: int, level: int, W: int, words: np.ndarray, exps: np.ndarray):
        w = np.ascontiguousarray(words, dtype=np.uint32)
        e = np.ascontiguousarray(exps, dtype=np.int8)
        self._chk(_lib.cmg_set_section(self._h, which, level, W, w.ctypes.data, e.ctypes.data),
                  "cmg_set_section")

    def decode_solution(self, z0: int = 0, nz: Optional[int] = None):
        import torch
        L = self.level
        n = (1 << L) - 1
        nzt = n if self.cfg.dim == 3 else 1
        if nz is None:
            nz = nzt - z0
        out = torch.empty((nz, n, n), dtype=torch.float64, device="cuda")
        self._chk(_lib.cmg_decode_solution(self._h, z0, nz, out.data_ptr()), "cmg_decode_solution")
        return out

    def state_save(self) -> bytes:
        ln = ctypes.c_size_t(0)
        self._chk(_lib.cmg_state_save(self._h, None, ctypes.byref(ln)), "cmg_state_save")
        buf = ctypes.create_string_buffer(ln.value)
        self._chk(_lib.cmg_state_save(self._h, buf, ctypes.byref(ln)), "cmg_state_save")
        return buf.raw[:ln.value]

    def state_load(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        self._chk(_lib.cmg_state_load(self._h, buf, len(data)), "cmg_state_load")


