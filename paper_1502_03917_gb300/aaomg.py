"""ctypes binding of the C ABI in ``include/aaomg.h`` (``libaaomg.so``).

Argument marshalling only: every step of the method runs in the CUDA library.
Vectors are torch float64 CUDA tensors (device calls) or numpy float64 arrays
(``solve_host``); the current torch CUDA stream is passed to every call.  If the
library is missing or no sm_103 GPU is present the calls raise -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libaaomg.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "aaomg.h")

SMOOTHER = {"ne": 0, "lsgs": 1, "slsgs": 2, "cgs": 3}
PRECISION = {"fp64": 0, "fp32_refine": 1}
CYCLE = {"V": 1, "W": 2}

OK, ERR_BAD_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_NO_DEVICE = 0, -1, -2, -3, -4, -5, -7

_lock = threading.Lock()
_lib = None


class MGError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [
        ("smoother", ctypes.c_int),
        ("nu_pre", ctypes.c_int),
        ("nu_post", ctypes.c_int),
        ("cycle", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("k_variant", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("inner_cycles", ctypes.c_int),
        ("coarse_level", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("tile_w", ctypes.c_int),
        ("tile_h", ctypes.c_int),
        ("small_max", ctypes.c_int),
        ("cluster_size", ctypes.c_int),
        ("profile_level", ctypes.c_int),
        ("autotune", ctypes.c_int),
    ]


def header_functions() -> list[str]:
    """Names of the functions the C header declares."""
    text = open(HEADER).read()
    return re.findall(r"AAOMG_API\s+[\w\s\*]+?\b(mg_\w+)\s*\(", text)


def load():
    """Load libaaomg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        H = ctypes.c_void_p
        I, D, P = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        pI, pD = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
        sig = {
            "mg_setup": (I, [I, D, ctypes.POINTER(Options), ctypes.POINTER(H)]),
            "mg_destroy": (None, [H]),
            "mg_num_nodes": (ctypes.c_longlong, [H]),
            "mg_rhs_from_yd": (I, [H, P, P, P]),
            "mg_residual": (I, [H, P, P, P, pD, P]),
            "mg_smooth": (I, [H, P, P, I, P]),
            "mg_restrict": (I, [H, P, P, P, P]),
            "mg_prolong_add": (I, [H, P, P, P]),
            "mg_cycle": (I, [H, P, P, P]),
            "mg_solve": (I, [H, P, P, D, pI, pD, P]),
            "mg_solve_host": (I, [H, P, P, D, pI, pD, P]),
            "mg_protocol_iterations": (I, [H, P, D, I, pI, P]),
            "mg_get_history": (I, [H, pD, I, pI]),
            "mg_norms": (I, [H, P, pD, pD, P]),
            "mg_level_kernel": (I, [H, I, pI, pI]),
            "mg_kernel_launches": (ctypes.c_longlong, [H]),
            "mg_get_profile": (I, [H, pD, ctypes.POINTER(ctypes.c_longlong)]),
            "mg_reset_profile": (I, [H]),
            "mg_residual_noalloc": (I, [I, D, I, P, P, P, pD, P]),
            "mg_solve_batch": (I, [I, ctypes.POINTER(H), ctypes.POINTER(P), ctypes.POINTER(P), D, pI, pD, P]),
            "mg_batch_create": (I, [I, ctypes.POINTER(H), ctypes.POINTER(H)]),
            "mg_batch_solve": (I, [H, ctypes.POINTER(P), ctypes.POINTER(P), D, pI, pD, pI, P]),
            "mg_batch_destroy": (None, [H]),
            "mg_batch_solve_host": (I, [H, ctypes.POINTER(P), ctypes.POINTER(P), D, pI, pD, pI, P]),
            "mg_batch_adjoint": (I, [H, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                     pD, D, pI, P]),
            "mg_control": (I, [H, P, P, P]),
            "mg_adjoint": (I, [H, P, P, P, P, pD, D, P]),
            "mg_device_peaks": (I, [pD, pD, pD, pD]),
            "mg_strerror": (ctypes.c_char_p, [I]),
            "mg_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(code: int, where: str, allow=()):
    if code != OK and code not in allow:
        lib = load()
        raise MGError(code, where, lib.mg_last_error().decode() or lib.mg_strerror(code).decode())
    return code


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t, n=None):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def device_peaks() -> dict:
    """The current device's FP32 and FP64 FMA rates (TFLOP/s), L2-resident read
    bandwidth and HBM copy bandwidth (GB/s), measured by mg_device_peaks."""
    lib = load()
    v = [ctypes.c_double() for _ in range(4)]
    _check(lib.mg_device_peaks(*[ctypes.byref(x) for x in v]), "mg_device_peaks")
    return {"fp32_tflops": v[0].value, "fp64_tflops": v[1].value, "l2_gbs": v[2].value, "hbm_copy_gbs": v[3].value}


def residual_noalloc(levels: int, alpha: float, f, x, r=None, k_variant: int = 0):
    """r = f - A x and the relative residual through mg_residual_noalloc: no
    handle and no device allocation inside the library (its scratch is a static
    device array; concurrent calls on different streams race)."""
    lib = load()
    N = ((1 << int(levels)) + 1) ** 2
    rr = ctypes.c_double()
    rp = _dptr(r, 2 * N) if r is not None else None
    code = lib.mg_residual_noalloc(int(levels), float(alpha), int(k_variant), _dptr(f, 2 * N), _dptr(x, 2 * N), rp,
                                   ctypes.byref(rr), _stream())
    if code != OK:
        # this entry point records no message: mg_last_error() would still hold
        # an earlier, unrelated failure of this thread
        raise MGError(code, "mg_residual_noalloc", lib.mg_strerror(code).decode())
    return rr.value


class Batch:
    """One graph-captured batch over several solvers (mg_batch_create): every
    solve() launches a single CUDA graph that runs each instance to its own
    convergence, the tests on the device.  The solvers must stay open while
    the batch is used."""

    def __init__(self, solvers):
        self._lib = load()
        self.solvers = list(solvers)
        n = len(self.solvers)
        hs = (ctypes.c_void_p * n)(*[s._h for s in self.solvers])
        b = ctypes.c_void_p()
        _check(self._lib.mg_batch_create(n, hs, ctypes.byref(b)), "mg_batch_create")
        self._b = b

    def solve(self, fs, xs, tol: float = 1e-8, raise_on_fail: bool = True):
        """Solve solvers[k] on (fs[k], xs[k]) for all k (xs in/out); returns
        (iterations, relative residuals, per-instance status, first status)."""
        n = len(self.solvers)
        fp = (ctypes.c_void_p * n)(*[_dptr(f, 2 * s.N) for s, f in zip(self.solvers, fs)])
        xp = (ctypes.c_void_p * n)(*[_dptr(x, 2 * s.N) for s, x in zip(self.solvers, xs)])
        it = (ctypes.c_int * n)()
        rr = (ctypes.c_double * n)()
        st = (ctypes.c_int * n)()
        code = self._lib.mg_batch_solve(self._b, fp, xp, float(tol), it, rr, st, _stream())
        if raise_on_fail:
            _check(code, "mg_batch_solve")
        return list(it), list(rr), list(st), code

    def solve_host(self, fs, xs, tol: float = 1e-8, raise_on_fail: bool = True):
        """solve() with fs and xs contiguous float64 numpy arrays in host
        memory (xs in/out): host-to-device and device-to-host copies inside."""
        import numpy as np

        n = len(self.solvers)
        for s, f, x in zip(self.solvers, fs, xs):
            for a in (f, x):
                if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                        and a.size == 2 * s.N):
                    raise TypeError("expected contiguous float64 numpy arrays of 2N elements")
        fp = (ctypes.c_void_p * n)(*[f.ctypes.data for f in fs])
        xp = (ctypes.c_void_p * n)(*[x.ctypes.data for x in xs])
        it = (ctypes.c_int * n)()
        rr = (ctypes.c_double * n)()
        st = (ctypes.c_int * n)()
        code = self._lib.mg_batch_solve_host(self._b, fp, xp, float(tol), it, rr, st, _stream())
        if raise_on_fail:
            _check(code, "mg_batch_solve_host")
        return list(it), list(rr), list(st), code

    def adjoint(self, xs, ubars, tol: float = 1e-10):
        """Batched mg_adjoint: for every instance the adjoint solve of the loss
        gradient ubars[k] = dL/du_k at the solution xs[k]; returns (gyD list,
        dL/dalpha list, z list, adjoint iterations)."""
        import torch

        n = len(self.solvers)
        zs = [torch.empty(2 * s.N, dtype=torch.float64, device=x.device) for s, x in zip(self.solvers, xs)]
        gs = [torch.empty(s.N, dtype=torch.float64, device=x.device) for s, x in zip(self.solvers, xs)]
        arr = lambda ts, m: (ctypes.c_void_p * n)(*[_dptr(t, m(s)) for s, t in zip(self.solvers, ts)])  # noqa: E731
        da = (ctypes.c_double * n)()
        it = (ctypes.c_int * n)()
        _check(self._lib.mg_batch_adjoint(self._b, arr(xs, lambda s: 2 * s.N), arr(ubars, lambda s: s.N),
                                          arr(zs, lambda s: 2 * s.N), arr(gs, lambda s: s.N), da, float(tol), it,
                                          _stream()), "mg_batch_adjoint")
        return gs, list(da), zs, list(it)

    def close(self):
        if getattr(self, "_b", None):
            self._lib.mg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def solve_batch(solvers, fs, xs, tol: float = 1e-8, raise_on_fail: bool = True):
    """Solve independent problems at once (mg_solve_batch: a one-shot batch
    graph): solvers[k] on (fs[k], xs[k]); returns (iterations, relative
    residuals, status)."""
    lib = load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s._h for s in solvers])
    fp = (ctypes.c_void_p * n)(*[_dptr(f, 2 * s.N) for s, f in zip(solvers, fs)])
    xp = (ctypes.c_void_p * n)(*[_dptr(x, 2 * s.N) for s, x in zip(solvers, xs)])
    it = (ctypes.c_int * n)()
    rr = (ctypes.c_double * n)()
    code = lib.mg_solve_batch(n, hs, fp, xp, float(tol), it, rr, _stream())
    if raise_on_fail:
        _check(code, "mg_solve_batch")
    return list(it), list(rr), code


class Solver:
    """One multigrid hierarchy (levels 1..L) for one alpha, owned by the library."""

    def __init__(self, levels: int, alpha: float, smoother: str = "lsgs", precision: str = "fp64",
                 cycle: str = "W", nu_pre: int = 0, nu_post: int = 0, tau: float = 0.0, k_variant: int = 0,
                 max_iter: int = 0, inner_cycles: int = 0, coarse_level: int = -1, profile: bool = False,
                 tile_w: int = 0, tile_h: int = 0, small_max: int = 0, cluster_size: int = 0,
                 profile_level: int = 0, autotune: bool = False):
        self._lib = load()
        self.levels, self.alpha = int(levels), float(alpha)
        self.smoother, self.precision, self.cycle_kind = smoother, precision, cycle
        opt = Options(SMOOTHER[smoother], int(nu_pre), int(nu_post), CYCLE[cycle], PRECISION[precision],
                      float(tau), int(k_variant), int(max_iter), int(inner_cycles), int(coarse_level),
                      int(bool(profile)), int(tile_w), int(tile_h), int(small_max), int(cluster_size),
                      int(profile_level), int(bool(autotune)))
        h = ctypes.c_void_p()
        _check(self._lib.mg_setup(self.levels, self.alpha, ctypes.byref(opt), ctypes.byref(h)), "mg_setup")
        self._h = h
        self.N = int(self._lib.mg_num_nodes(h))
        self.nc = ((1 << (self.levels - 1)) + 1) ** 2 if self.levels > 1 else 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- device calls ------------------------------------------------------
    def rhs_from_yd(self, yD, f=None):
        import torch

        f = torch.empty(2 * self.N, dtype=torch.float64, device=yD.device) if f is None else f
        _check(self._lib.mg_rhs_from_yd(self._h, _dptr(yD, self.N), _dptr(f, 2 * self.N), _stream()), "mg_rhs_from_yd")
        return f

    def residual(self, f, x, r=None):
        rr = ctypes.c_double()
        rp = _dptr(r, 2 * self.N) if r is not None else None
        _check(self._lib.mg_residual(self._h, _dptr(f, 2 * self.N), _dptr(x, 2 * self.N), rp, ctypes.byref(rr),
                                     _stream()), "mg_residual")
        return rr.value

    def smooth(self, f, x, steps: int = 1):
        _check(self._lib.mg_smooth(self._h, _dptr(f, 2 * self.N), _dptr(x, 2 * self.N), int(steps), _stream()),
               "mg_smooth")
        return x

    def restrict(self, f, x, fc=None):
        import torch

        fc = torch.empty(2 * self.nc, dtype=torch.float64, device=f.device) if fc is None else fc
        _check(self._lib.mg_restrict(self._h, _dptr(f, 2 * self.N), _dptr(x, 2 * self.N), _dptr(fc, 2 * self.nc),
                                     _stream()), "mg_restrict")
        return fc

    def prolong_add(self, xc, x):
        _check(self._lib.mg_prolong_add(self._h, _dptr(xc, 2 * self.nc), _dptr(x, 2 * self.N), _stream()),
               "mg_prolong_add")
        return x

    def cycle(self, f, x):
        _check(self._lib.mg_cycle(self._h, _dptr(f, 2 * self.N), _dptr(x, 2 * self.N), _stream()), "mg_cycle")
        return x

    def solve(self, f, x, tol: float = 1e-8, raise_on_fail: bool = True):
        it, rr = ctypes.c_int(), ctypes.c_double()
        code = self._lib.mg_solve(self._h, _dptr(f, 2 * self.N), _dptr(x, 2 * self.N), float(tol), ctypes.byref(it),
                                  ctypes.byref(rr), _stream())
        if raise_on_fail:
            _check(code, "mg_solve")
        return it.value, rr.value, code

    def level_kernels(self):
        """{level: (kind, blocks)} for levels 1..L: kind 'phases', 'strips',
        'band' or 'coarse', blocks as returned by mg_level_kernel."""
        names = {0: "phases", 1: "strips", 2: "band", 3: "coarse"}
        out = {}
        for l in range(1, self.levels + 1):
            k, b = ctypes.c_int(), ctypes.c_int()
            _check(self._lib.mg_level_kernel(self._h, l, ctypes.byref(k), ctypes.byref(b)), "mg_level_kernel")
            out[l] = (names[k.value], b.value)
        return out

    def norms(self, x):
        """(||x||_L, ||x||_{L^-1}) on the finest level (the paper's L = diag(Q))."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(self._lib.mg_norms(self._h, _dptr(x, 2 * self.N), ctypes.byref(a), ctypes.byref(b), _stream()),
               "mg_norms")
        return a.value, b.value

    def protocol_iterations(self, x0, reduction: float = 1e-6, max_iter: int = 300) -> int:
        """Section 3's protocol (mg_protocol_iterations): zero right-hand side,
        start x0 (not modified), cycles until ||x||_L has dropped by
        `reduction`; -1 if max_iter is hit."""
        it = ctypes.c_int()
        code = self._lib.mg_protocol_iterations(self._h, _dptr(x0, 2 * self.N), float(reduction), int(max_iter),
                                                ctypes.byref(it), _stream())
        _check(code, "mg_protocol_iterations", allow=(ERR_NOT_CONVERGED,))
        return it.value

    def solve_host(self, f, x, tol: float = 1e-8, raise_on_fail: bool = True):
        """f, x: C-contiguous float64 numpy arrays (x in/out) in host memory."""
        import numpy as np

        for a in (f, x):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.size == 2 * self.N):
                raise TypeError("expected contiguous float64 numpy arrays of 2N elements")
        if not x.flags.writeable:
            raise ValueError("x must be writeable")
        it, rr = ctypes.c_int(), ctypes.c_double()
        code = self._lib.mg_solve_host(self._h, ctypes.c_void_p(f.ctypes.data), ctypes.c_void_p(x.ctypes.data),
                                       float(tol), ctypes.byref(it), ctypes.byref(rr), _stream())
        if raise_on_fail:
            _check(code, "mg_solve_host")
        return it.value, rr.value, code

    def control(self, x, u=None):
        """u = lambda / alpha of x = (y, lambda)."""
        import torch

        u = torch.empty(self.N, dtype=torch.float64, device=x.device) if u is None else u
        _check(self._lib.mg_control(self._h, _dptr(x, 2 * self.N), _dptr(u, self.N), _stream()), "mg_control")
        return u

    def adjoint(self, x, ubar, tol: float = 1e-10):
        """(gyD, dL/dalpha, z) for a loss of the control u = lambda/alpha, given
        the solution x and ubar = dL/du (see mg_adjoint)."""
        import torch

        z = torch.empty(2 * self.N, dtype=torch.float64, device=x.device)
        gyD = torch.empty(self.N, dtype=torch.float64, device=x.device)
        da = ctypes.c_double()
        _check(self._lib.mg_adjoint(self._h, _dptr(x, 2 * self.N), _dptr(ubar, self.N), _dptr(z, 2 * self.N),
                                    _dptr(gyD, self.N), ctypes.byref(da), float(tol), _stream()), "mg_adjoint")
        return gyD, da.value, z

    def history(self):
        buf = (ctypes.c_double * 1024)()
        n = ctypes.c_int()
        _check(self._lib.mg_get_history(self._h, buf, 1024, ctypes.byref(n)), "mg_get_history")
        return [buf[i] for i in range(n.value)]

    def profile(self):
        """(ms, sweeps): device time of the smoothing calls on the profiled
        level (the finest unless profile_level is set) inside the iterations
        since the last reset, and the sweeps they cover."""
        ms, sw = ctypes.c_double(), ctypes.c_longlong()
        _check(self._lib.mg_get_profile(self._h, ctypes.byref(ms), ctypes.byref(sw)), "mg_get_profile")
        return ms.value, sw.value

    def reset_profile(self):
        _check(self._lib.mg_reset_profile(self._h), "mg_reset_profile")

    def launches(self) -> int:
        return int(self._lib.mg_kernel_launches(self._h))
