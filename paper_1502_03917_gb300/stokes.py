"""ctypes binding of the Stokes control entry points (``include/aaomg_stokes.h``)
in ``libaaomg.so``.

Argument marshalling only: every step of the method runs in the CUDA library.
Vectors are contiguous float64 CUDA tensors in the block order
``(v_1, v_2, p, lambda_1, lambda_2, mu)``; the current torch CUDA stream is
passed to every call.  Without the built library or an sm_103 GPU the calls
raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import aaomg as _mg

HEADER = os.path.join(os.path.dirname(_mg.PKG), "include", "aaomg_stokes.h")
SMOOTHER = {"ne": 0, "lsgs": 1, "slsgs": 2}
CYCLE = {"V": 1, "W": 2}

_lock = threading.Lock()
_ready = False


class Options(ctypes.Structure):
    _fields_ = [
        ("smoother", ctypes.c_int),
        ("nu_pre", ctypes.c_int),
        ("nu_post", ctypes.c_int),
        ("cycle", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("block_max", ctypes.c_int),
        ("dense_level", ctypes.c_int),
    ]


def header_functions() -> list[str]:
    """Names of the functions the Stokes header declares."""
    return re.findall(r"AAOMG_API\s+[\w\s\*]+?\b(ms_\w+)\s*\(", open(HEADER).read())


def load():
    global _ready
    lib = _mg.load()
    with _lock:
        if _ready:
            return lib
        H, I, D, P = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        pI, pD = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
        sig = {
            "ms_setup": (I, [I, D, ctypes.POINTER(Options), ctypes.POINTER(H)]),
            "ms_destroy": (None, [H]),
            "ms_sizes": (I, [H, I, pI]),
            "ms_rhs_from_vd": (I, [H, P, P, P]),
            "ms_residual": (I, [H, P, P, P, pD, P]),
            "ms_smooth": (I, [H, P, P, I, P]),
            "ms_cycle": (I, [H, P, P, P]),
            "ms_solve": (I, [H, P, P, D, pI, pD, P]),
            "ms_normalize": (I, [H, P, P]),
            "ms_control": (I, [H, P, P, P]),
            "ms_norms": (I, [H, P, pD, pD, P]),
            "ms_protocol_iterations": (I, [H, P, D, I, pI, P]),
            "ms_kernel_launches": (ctypes.c_longlong, [H]),
            "ms_operator_entries": (I, [H, I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _ready = True
        return lib


class StokesSolver:
    """One hierarchy (levels 1..L, h = 2^-L finest) for one alpha."""

    def __init__(self, levels: int, alpha: float, smoother: str = "lsgs", cycle: str = "W", nu_pre: int = 0,
                 nu_post: int = 0, tau: float = 0.0, max_iter: int = 0, block_max: int = 0,
                 dense_level: int = 0):
        self._lib = load()
        self.levels, self.alpha, self.smoother = int(levels), float(alpha), smoother
        opt = Options(SMOOTHER[smoother], int(nu_pre), int(nu_post), CYCLE[cycle], float(tau), int(max_iter),
                      int(block_max), int(dense_level))
        h = ctypes.c_void_p()
        _mg._check(self._lib.ms_setup(self.levels, self.alpha, ctypes.byref(opt), ctypes.byref(h)), "ms_setup")
        self._h = h
        s = self.sizes()
        self.n, self.nv, self.np, self.m = s

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ms_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sizes(self, level: int | None = None):
        out = (ctypes.c_int * 4)()
        _mg._check(self._lib.ms_sizes(self._h, self.levels if level is None else int(level), out), "ms_sizes")
        return tuple(int(v) for v in out)

    def rhs_from_vd(self, vD, f=None):
        import torch

        ng2 = (2 * self.n + 1) ** 2
        f = torch.empty(self.m, dtype=torch.float64, device=vD.device) if f is None else f
        _mg._check(self._lib.ms_rhs_from_vd(self._h, _mg._dptr(vD, 2 * ng2), _mg._dptr(f, self.m), _mg._stream()),
                   "ms_rhs_from_vd")
        return f

    def residual(self, f, x, r=None):
        rr = ctypes.c_double()
        rp = _mg._dptr(r, self.m) if r is not None else None
        _mg._check(self._lib.ms_residual(self._h, _mg._dptr(f, self.m), _mg._dptr(x, self.m), rp, ctypes.byref(rr),
                                         _mg._stream()), "ms_residual")
        return rr.value

    def smooth(self, f, x, steps: int = 1):
        _mg._check(self._lib.ms_smooth(self._h, _mg._dptr(f, self.m), _mg._dptr(x, self.m), int(steps),
                                       _mg._stream()), "ms_smooth")

    def cycle(self, f, x):
        _mg._check(self._lib.ms_cycle(self._h, _mg._dptr(f, self.m), _mg._dptr(x, self.m), _mg._stream()),
                   "ms_cycle")

    def solve(self, f, x, tol: float = 1e-8, raise_on_fail: bool = True):
        it, rr = ctypes.c_int(), ctypes.c_double()
        code = self._lib.ms_solve(self._h, _mg._dptr(f, self.m), _mg._dptr(x, self.m), float(tol), ctypes.byref(it),
                                  ctypes.byref(rr), _mg._stream())
        if raise_on_fail:
            _mg._check(code, "ms_solve")
        return it.value, rr.value, code

    def normalize(self, x):
        _mg._check(self._lib.ms_normalize(self._h, _mg._dptr(x, self.m), _mg._stream()), "ms_normalize")

    def control(self, x, u=None):
        """u = lambda / alpha (both components on the interior P2 nodes)."""
        import torch

        u = torch.empty(2 * self.nv, dtype=torch.float64, device=x.device) if u is None else u
        _mg._check(self._lib.ms_control(self._h, _mg._dptr(x, self.m), _mg._dptr(u, 2 * self.nv), _mg._stream()),
                   "ms_control")
        return u

    def norms(self, x):
        nl, ni = ctypes.c_double(), ctypes.c_double()
        _mg._check(self._lib.ms_norms(self._h, _mg._dptr(x, self.m), ctypes.byref(nl), ctypes.byref(ni),
                                      _mg._stream()), "ms_norms")
        return nl.value, ni.value

    def protocol_iterations(self, x0, reduction: float = 1e-6, max_iter: int = 200) -> int:
        it = ctypes.c_int()
        _mg._check(self._lib.ms_protocol_iterations(self._h, _mg._dptr(x0, self.m), float(reduction), int(max_iter),
                                                    ctypes.byref(it), _mg._stream()), "ms_protocol_iterations")
        return it.value

    def kernel_launches(self) -> int:
        return int(self._lib.ms_kernel_launches(self._h))

    def operator_entries(self, level: int | None = None):
        """(nonzeros of A, entries held) on a level (the finest by default)."""
        nnz, stored = ctypes.c_longlong(), ctypes.c_longlong()
        _mg._check(self._lib.ms_operator_entries(self._h, self.levels if level is None else int(level),
                                                 ctypes.byref(nnz), ctypes.byref(stored)), "ms_operator_entries")
        return nnz.value, stored.value
