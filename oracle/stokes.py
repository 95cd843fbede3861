"""Plain FP64 CPU oracle for the all-at-once multigrid method applied to the
Stokes control problem (Takacs, "Efficient smoothers for all-at-once multigrid
methods for Poisson and Stokes control problems": section 1, second model
problem, eq. (mp3); section 2; section 3 and Table 2).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by ``bench.py``'s CPU
legs, never by the product package.  It shares no code with the CUDA library.
The arithmetic lives in ``stokes_oracle.c`` (built with gcc on first use); this
module only marshals numpy arrays through ctypes.

Unknowns of level k (n = 2^k cells per side, h = 1/n), in this order:
``x = (v_1, v_2, p, lambda_1, lambda_2, mu)``.  Velocities live on the
interior nodes of the P2 half-step grid (node (a, b) at (a h/2, b h/2),
1 <= a, b <= 2n-1, index (b-1)(2n-1) + (a-1)); pressures on all P1 vertices
(node (i, j) at (i h, j h), index j(n+1) + i).

* ``csr(level, which)`` -- the P2 mass ``M`` and stiffness ``K`` (interior
  nodes, one velocity component), the divergence blocks ``Dx``, ``Dy``
  ((D v)_q = -int psi_q div v), ``A`` of eq. (mp3), the embeddings ``P2`` and
  ``P1`` from level-1, and the full P2 matrices ``Mf``, ``Kf``, ``Dxf``, ``Dyf``
  over all (2n+1)^2 half-step nodes.
* ``ldiag`` -- L_k of section 2 for the Stokes problem; ``ndiag`` -- N_ii.
* ``smooth`` -- Algorithm 1 (NE, tau = 0.35 by default), Algorithm 2 (LSGS),
  sLSGS; ``cycle`` / ``solve`` -- the multigrid of section 2;
  ``protocol_iterations`` -- section 3.
* ``normalize`` -- removes the means of p and mu (the paper's int p = 0).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stokes_oracle.c")
_LIB = os.path.join(_HERE, "libstokes_oracle.so")
_lock = threading.Lock()
_lib = None

SMOOTHERS = {"ne": 0, "lsgs": 1, "slsgs": 2}
_WHICH = {"M": 0, "K": 1, "Dx": 2, "Dy": 3, "A": 4, "P2": 5, "P1": 6, "Mf": 7, "Kf": 8, "Dxf": 9, "Dyf": 10}
VCOL, PCOL = 19, 7  # colours of the multicolour order (P2 half-step grid, P1 vertices)


def build(force: bool = False) -> str:
    """Compile ``oracle/libstokes_oracle.so`` (plain C, -O2, no FMA contraction)."""
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
        P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
        sig = {
            "sto_create": (P, [I, D, I, I, I, I, D, I]),
            "sto_destroy": (None, [P]),
            "sto_sizes": (None, [P, I, ip]),
            "sto_csr_nnz": (ctypes.c_int64, [P, I, I]),
            "sto_csr_shape": (None, [P, I, I, ip]),
            "sto_csr_export": (None, [P, I, I, lp, ip, dp]),
            "sto_ldiag": (None, [P, I, dp]),
            "sto_ndiag": (None, [P, I, dp]),
            "sto_order": (None, [P, I, ip]),
            "sto_pweights": (None, [P, I, dp]),
            "sto_rhs": (None, [P, dp, dp]),
            "sto_residual": (None, [P, I, dp, dp, dp]),
            "sto_normalize": (None, [P, I, dp]),
            "sto_norm_Linv": (D, [P, I, dp]),
            "sto_norm_L": (D, [P, I, dp]),
            "sto_smooth": (None, [P, I, dp, dp, I]),
            "sto_restrict": (None, [P, I, dp, dp]),
            "sto_prolong_add": (None, [P, I, dp, dp]),
            "sto_coarse_solve": (None, [P, dp, dp]),
            "sto_cycle": (None, [P, I, dp, dp]),
            "sto_solve": (I, [P, dp, dp, D, I, ctypes.POINTER(D), dp]),
            "sto_protocol_iterations": (I, [P, dp, D, I]),
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


class StokesOracle:
    """One hierarchy (levels 1..L, h_k = 2^-k, coarsest h = 1/2) for one alpha."""

    def __init__(self, L: int, alpha: float, smoother: str = "lsgs", nu_pre: int = 2, nu_post: int = 2,
                 gamma: int = 2, tau: float = 0.35, lexicographic: bool = False):
        self._lib = _load()
        self.L, self.alpha, self.smoother = int(L), float(alpha), smoother
        self._h = self._lib.sto_create(self.L, self.alpha, SMOOTHERS[smoother], int(nu_pre), int(nu_post),
                                       int(gamma), float(tau), int(bool(lexicographic)))
        if not self._h:
            raise ValueError(f"stokes oracle: bad arguments L={L} alpha={alpha}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sto_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _lev(self, level):
        return self.L if level is None else int(level)

    def sizes(self, level: int | None = None) -> dict:
        """n (cells per side), nv (unknowns per velocity component), np (P1
        vertices), m (all unknowns) and the block offsets of x."""
        out = np.empty(4, np.int32)
        self._lib.sto_sizes(self._h, self._lev(level), out)
        n, nv, npn, m = (int(v) for v in out)
        return {"n": n, "nv": nv, "np": npn, "m": m,
                "v": (0, nv), "p": 2 * nv, "l": (2 * nv + npn, 3 * nv + npn), "mu": 4 * nv + npn}

    def m(self, level: int | None = None) -> int:
        return self.sizes(level)["m"]

    # -- matrices -----------------------------------------------------------
    def csr(self, level: int, which: str):
        w = _WHICH[which]
        shape = np.empty(2, np.int32)
        self._lib.sto_csr_shape(self._h, level, w, shape)
        nnz = self._lib.sto_csr_nnz(self._h, level, w)
        rp = np.empty(int(shape[0]) + 1, np.int64)
        col = np.empty(max(nnz, 1), np.int32)
        val = np.empty(max(nnz, 1), np.float64)
        self._lib.sto_csr_export(self._h, level, w, rp, col, val)
        return rp, col[:nnz], val[:nnz], (int(shape[0]), int(shape[1]))

    def scipy(self, level: int, which: str):
        import scipy.sparse as sp

        rp, col, val, shape = self.csr(level, which)
        return sp.csr_matrix((val, col, rp), shape=shape)

    def ldiag(self, level: int | None = None) -> np.ndarray:
        level = self._lev(level)
        out = np.empty(self.m(level))
        self._lib.sto_ldiag(self._h, level, out)
        return out

    def ndiag(self, level: int | None = None) -> np.ndarray:
        level = self._lev(level)
        out = np.empty(self.m(level))
        self._lib.sto_ndiag(self._h, level, out)
        return out

    def order(self, level: int | None = None) -> np.ndarray:
        level = self._lev(level)
        out = np.empty(self.m(level), np.int32)
        self._lib.sto_order(self._h, level, out)
        return out

    def pweights(self, level: int | None = None) -> np.ndarray:
        """int psi_q for every P1 vertex q (sums to |Omega| = 1)."""
        level = self._lev(level)
        out = np.empty(self.sizes(level)["np"])
        self._lib.sto_pweights(self._h, level, out)
        return out

    # -- vectors ------------------------------------------------------------
    def rhs(self, vD) -> np.ndarray:
        """f = (M v_D, 0, 0, 0); vD: both components at all (2n+1)^2 P2 nodes,
        component-major (length 2 (2n+1)^2)."""
        s = self.sizes()
        ng2 = (2 * s["n"] + 1) ** 2
        f = np.empty(s["m"])
        self._lib.sto_rhs(self._h, _f64(vD, 2 * ng2), f)
        return f

    def residual(self, f, x, level: int | None = None) -> np.ndarray:
        level = self._lev(level)
        m = self.m(level)
        r = np.empty(m)
        self._lib.sto_residual(self._h, level, _f64(f, m), _f64(x, m), r)
        return r

    def normalize(self, x, level: int | None = None) -> np.ndarray:
        level = self._lev(level)
        x = _f64(x, self.m(level)).copy()
        self._lib.sto_normalize(self._h, level, x)
        return x

    def norm_Linv(self, v, level: int | None = None) -> float:
        level = self._lev(level)
        return self._lib.sto_norm_Linv(self._h, level, _f64(v, self.m(level)))

    def norm_L(self, v, level: int | None = None) -> float:
        level = self._lev(level)
        return self._lib.sto_norm_L(self._h, level, _f64(v, self.m(level)))

    def smooth(self, f, x, steps: int = 1, level: int | None = None) -> np.ndarray:
        level = self._lev(level)
        m = self.m(level)
        x = _f64(x, m).copy()
        self._lib.sto_smooth(self._h, level, _f64(f, m), x, int(steps))
        return x

    def restrict(self, rf, level: int | None = None) -> np.ndarray:
        level = self._lev(level)
        rc = np.empty(self.m(level - 1))
        self._lib.sto_restrict(self._h, level, _f64(rf, self.m(level)), rc)
        return rc

    def prolong_add(self, xc, xf, level: int | None = None) -> np.ndarray:
        level = self._lev(level)
        xf = _f64(xf, self.m(level)).copy()
        self._lib.sto_prolong_add(self._h, level, _f64(xc, self.m(level - 1)), xf)
        return xf

    def coarse_solve(self, f) -> np.ndarray:
        m = self.m(1)
        x = np.empty(m)
        self._lib.sto_coarse_solve(self._h, _f64(f, m), x)
        return x

    def cycle(self, f, x, level: int | None = None) -> np.ndarray:
        level = self._lev(level)
        m = self.m(level)
        x = _f64(x, m).copy()
        self._lib.sto_cycle(self._h, level, _f64(f, m), x)
        return x

    def solve(self, f, x0=None, tol: float = 1e-8, max_iter: int = 100):
        """(x, iterations, relative residual in ||.||_{L^-1}, history)."""
        m = self.m()
        x = np.zeros(m) if x0 is None else _f64(x0, m).copy()
        rr = ctypes.c_double()
        hist = np.zeros(max_iter + 1)
        it = self._lib.sto_solve(self._h, _f64(f, m), x, float(tol), int(max_iter), ctypes.byref(rr), hist)
        return x, it, rr.value, hist[: it + 1]

    def protocol_iterations(self, x0, reduction: float = 1e-6, max_iter: int = 200) -> int:
        x = _f64(x0, self.m()).copy()
        return int(self._lib.sto_protocol_iterations(self._h, x, float(reduction), int(max_iter)))
