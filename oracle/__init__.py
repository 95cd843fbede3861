"""Plain FP64 CPU oracle for the all-at-once multigrid method (Poisson control).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
(as the checker) and by ``bench.py``'s CPU-baseline leg, never by the product
package.  It shares no code with the CUDA library.  The arithmetic lives in
``aaomg_oracle.c`` (built with gcc on first use); this module only marshals
numpy arrays through ctypes.

What each call computes, with its source in the paper (Takacs, "Efficient
smoothers for all-at-once multigrid methods for Poisson and Stokes control
problems"):

* ``Oracle.csr(level, 'M'|'K'|'A'|'P')`` -- P1 mass/stiffness matrices by
  element loops, A_k of eq. (mp2), the canonical embedding I_{k-1}^k (section 2).
* ``ldiag`` -- L_k = diag(Q_k), section 2; ``ndiag`` -- N_ii of Algorithm 2.
* ``smooth`` -- Algorithm 1 (NE), Algorithm 2 (LSGS), sLSGS, CGS (section 2).
* ``restrict`` / ``prolong_add`` -- I_k^{k-1} = (I_{k-1}^k)^T and I_{k-1}^k.
* ``cycle`` / ``solve`` -- the multigrid iteration of section 2 (V or W).
* ``protocol_iterations`` -- the iteration count protocol of section 3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aaomg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SMOOTHERS = {"ne": 0, "lsgs": 1, "slsgs": 2, "cgs": 3}
_WHICH = {"M": 0, "K": 1, "A": 2, "P": 3}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain C, -O2, no FMA
    contraction so that results are identical on every host)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        D = ctypes.c_double
        I = ctypes.c_int
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
        sig = {
            "or_create": (P, [I, D, I, I, I, I, I, D, I]),
            "or_destroy": (None, [P]),
            "or_nnodes": (I, [P, I]),
            "or_csr_nnz": (ctypes.c_int64, [P, I, I]),
            "or_csr_shape": (I, [P, I, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
            "or_csr_export": (None, [P, I, I, lp, ip, dp]),
            "or_ldiag": (None, [P, I, dp]),
            "or_ndiag": (None, [P, I, dp]),
            "or_order": (None, [P, I, ip]),
            "or_rhs": (None, [P, dp, dp]),
            "or_residual": (None, [P, I, dp, dp, dp]),
            "or_norm_Linv": (D, [P, I, dp]),
            "or_norm_L": (D, [P, I, dp]),
            "or_smooth": (None, [P, I, dp, dp, I]),
            "or_restrict": (None, [P, I, dp, dp]),
            "or_prolong_add": (None, [P, I, dp, dp]),
            "or_coarse_solve": (None, [P, dp, dp]),
            "or_cycle": (None, [P, I, dp, dp]),
            "or_solve": (I, [P, dp, dp, D, I, ctypes.POINTER(D), dp]),
            "or_protocol_iterations": (I, [P, dp, D, I]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.shape != (n,):
        raise ValueError(f"expected shape ({n},), got {a.shape}")
    return a


class Oracle:
    """One multigrid hierarchy (levels 1..L, h_k = 2^-k) for one alpha.

    Unknowns per level: x = (y, lambda), each of (2^k+1)^2 nodal values stored
    row by row (index j*(n+1)+i for node (i h, j h)).
    """

    def __init__(self, L: int, alpha: float, smoother: str = "lsgs", nu_pre: int = 2, nu_post: int = 2,
                 gamma: int = 2, tau: float = 0.4, kvariant: int = 0, lexicographic: bool = False):
        self._lib = _load()
        self.L, self.alpha = int(L), float(alpha)
        self.smoother = smoother
        self._h = self._lib.or_create(self.L, self.alpha, int(kvariant), SMOOTHERS[smoother], int(nu_pre),
                                      int(nu_post), int(gamma), float(tau), int(bool(lexicographic)))
        if not self._h:
            raise ValueError(f"oracle: bad arguments L={L} alpha={alpha}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.or_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def nn(self, level: int | None = None) -> int:
        return self._lib.or_nnodes(self._h, self.L if level is None else level)

    # -- matrices -----------------------------------------------------------
    def csr(self, level: int, which: str):
        """(indptr, indices, data, shape) of M, K, A or P on `level`."""
        w = _WHICH[which]
        nr, nc = ctypes.c_int(), ctypes.c_int()
        self._lib.or_csr_shape(self._h, level, w, ctypes.byref(nr), ctypes.byref(nc))
        nnz = self._lib.or_csr_nnz(self._h, level, w)
        rp = np.empty(nr.value + 1, np.int64)
        col = np.empty(max(nnz, 1), np.int32)
        val = np.empty(max(nnz, 1), np.float64)
        self._lib.or_csr_export(self._h, level, w, rp, col, val)
        return rp, col[:nnz], val[:nnz], (nr.value, nc.value)

    def scipy(self, level: int, which: str):
        import scipy.sparse as sp

        rp, col, val, shape = self.csr(level, which)
        return sp.csr_matrix((val, col, rp), shape=shape)

    def ldiag(self, level: int | None = None) -> np.ndarray:
        level = self.L if level is None else level
        out = np.empty(2 * self.nn(level))
        self._lib.or_ldiag(self._h, level, out)
        return out

    def ndiag(self, level: int | None = None) -> np.ndarray:
        level = self.L if level is None else level
        out = np.empty(2 * self.nn(level))
        self._lib.or_ndiag(self._h, level, out)
        return out

    def order(self, level: int | None = None) -> np.ndarray:
        level = self.L if level is None else level
        out = np.empty(2 * self.nn(level), np.int32)
        self._lib.or_order(self._h, level, out)
        return out

    # -- vectors ------------------------------------------------------------
    def rhs(self, yD) -> np.ndarray:
        n = self.nn()
        f = np.empty(2 * n)
        self._lib.or_rhs(self._h, _f64(yD, n), f)
        return f

    def residual(self, f, x, level: int | None = None) -> np.ndarray:
        level = self.L if level is None else level
        n2 = 2 * self.nn(level)
        r = np.empty(n2)
        self._lib.or_residual(self._h, level, _f64(f, n2), _f64(x, n2), r)
        return r

    def norm_Linv(self, v, level: int | None = None) -> float:
        level = self.L if level is None else level
        return self._lib.or_norm_Linv(self._h, level, _f64(v, 2 * self.nn(level)))

    def norm_L(self, v, level: int | None = None) -> float:
        level = self.L if level is None else level
        return self._lib.or_norm_L(self._h, level, _f64(v, 2 * self.nn(level)))

    def smooth(self, f, x, steps: int = 1, level: int | None = None) -> np.ndarray:
        level = self.L if level is None else level
        n2 = 2 * self.nn(level)
        x = _f64(x, n2).copy()
        self._lib.or_smooth(self._h, level, _f64(f, n2), x, int(steps))
        return x

    def restrict(self, rf, level: int | None = None) -> np.ndarray:
        level = self.L if level is None else level
        rc = np.empty(2 * self.nn(level - 1))
        self._lib.or_restrict(self._h, level, _f64(rf, 2 * self.nn(level)), rc)
        return rc

    def prolong_add(self, xc, xf, level: int | None = None) -> np.ndarray:
        level = self.L if level is None else level
        xf = _f64(xf, 2 * self.nn(level)).copy()
        self._lib.or_prolong_add(self._h, level, _f64(xc, 2 * self.nn(level - 1)), xf)
        return xf

    def coarse_solve(self, f) -> np.ndarray:
        x = np.empty(2 * self.nn(1))
        self._lib.or_coarse_solve(self._h, _f64(f, 2 * self.nn(1)), x)
        return x

    def cycle(self, f, x, level: int | None = None) -> np.ndarray:
        level = self.L if level is None else level
        n2 = 2 * self.nn(level)
        x = _f64(x, n2).copy()
        self._lib.or_cycle(self._h, level, _f64(f, n2), x)
        return x

    def solve(self, f, x0=None, tol: float = 1e-8, max_iter: int = 200):
        """Returns (x, iterations, relres, history)."""
        n2 = 2 * self.nn()
        x = np.zeros(n2) if x0 is None else _f64(x0, n2).copy()
        hist = np.empty(max_iter + 1)
        rr = ctypes.c_double()
        it = self._lib.or_solve(self._h, _f64(f, n2), x, float(tol), int(max_iter), ctypes.byref(rr), hist)
        return x, it, rr.value, hist[: it + 1].copy()

    def protocol_iterations(self, x0, reduction: float = 1e-6, max_iter: int = 200) -> int:
        x = _f64(x0, 2 * self.nn()).copy()
        return self._lib.or_protocol_iterations(self._h, x, float(reduction), int(max_iter))
