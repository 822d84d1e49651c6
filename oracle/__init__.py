"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
it is plain C (``oracle.c``, compiled to ``liboracle.so`` with gcc) behind
ctypes, and it reads the same seeded inputs from :mod:`synth`.

Every function follows the DuaLip-GPU technical report (arXiv 2603.04621):
the smoothed dual and its Danskin gradient (Section 3.1, Eq. 2), the
per-source simplex projection (Section 3.2, Eqs. 4-5), Jacobi row
normalisation and primal scaling (Section 5.1), gamma continuation
(Section 5.1, Section 7) and the capped-step accelerated ascent (Appendix B).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
TRACE_W = 8


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
            _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class SolveOpts(ctypes.Structure):
    _fields_ = [("gamma0", ctypes.c_double), ("gamma_final", ctypes.c_double),
                ("halve_every", ctypes.c_int32), ("max_step", ctypes.c_double),
                ("init_step", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("tol_gap", ctypes.c_double), ("tol_infeas", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("row_normalize", ctypes.c_int32),
                ("restart_on_gamma_change", ctypes.c_int32), ("stop_on_tol", ctypes.c_int32),
                ("restart_on_decrease", ctypes.c_int32)]


class SolveResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("dual", ctypes.c_double), ("primal_lin", ctypes.c_double),
                ("reg", ctypes.c_double), ("infeas", ctypes.c_double),
                ("gap_rel", ctypes.c_double), ("infeas_rel", ctypes.c_double),
                ("gamma", ctypes.c_double), ("restarts", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.oracle_create.restype = vp
        lib.oracle_create.argtypes = [i64, i32, vp, vp, vp, vp, vp, ctypes.c_int]
        lib.oracle_create_multi.restype = vp
        lib.oracle_create_multi.argtypes = [i64, i32, i32, vp, vp, vp, vp, vp, ctypes.c_int]
        lib.oracle_destroy.argtypes = [vp]
        lib.oracle_project.argtypes = [i64, vp, vp, ctypes.c_int, vp, vp]
        lib.oracle_row_scale.argtypes = [vp, vp]
        lib.oracle_norm2_sq.argtypes = [vp, vp]
        lib.oracle_norm2_sq.restype = dbl
        lib.oracle_eval.argtypes = [vp, vp, dbl, ctypes.c_int, vp, vp, vp, vp]
        lib.oracle_solve.argtypes = [vp, ctypes.POINTER(SolveOpts), vp,
                                     ctypes.POINTER(SolveResult), vp]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_box.argtypes = [vp, ctypes.c_int]
        lib.oracle_set_box.restype = None
        _lib = lib
    return _lib


def _p(x):
    return None if x is None else ctypes.c_void_p(x.ctypes.data)


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 = leave); returns the count in use."""
    return int(_load().oracle_set_threads(n))


def project(r, alpha, method: str = "sort"):
    """x = alpha * (r - tau)_+ with tau >= 0 the multiplier of sum x <= 1
    (weighted Euclidean projection onto {x >= 0, sum x <= 1})."""
    lib = _load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    alpha = np.ascontiguousarray(np.broadcast_to(alpha, r.shape), dtype=np.float64)
    x = np.empty_like(r)
    tau = ctypes.c_double(0.0)
    rc = lib.oracle_project(r.shape[0], _p(r), _p(alpha), 0 if method == "sort" else 1, _p(x),
                            ctypes.byref(tau))
    if rc:
        raise RuntimeError(f"oracle_project failed ({rc})")
    return x, tau.value


@dataclass
class Eval:
    dual: float
    primal_lin: float
    reg: float
    infeas: float
    mu_dot_grad: float
    grad: np.ndarray
    ax: np.ndarray
    x: np.ndarray | None


class Problem:
    """One matching LP held by the oracle (keeps references to the arrays)."""

    def __init__(self, inst, weighted: bool = False, box: bool = False):
        """``inst.a`` is [E] (one constraint family) or [m, E] (m families,
        Definition 1); ``inst.b`` then has m J entries, row k J + j."""
        self._lib = _load()
        self.inst = inst
        a = np.asarray(inst.a, dtype=np.float32)
        self.m = 1 if a.ndim == 1 else int(a.shape[0])
        self._keep = [np.ascontiguousarray(inst.off, dtype=np.int64),
                      np.ascontiguousarray(inst.dst, dtype=np.int32),
                      np.ascontiguousarray(inst.c, dtype=np.float32),
                      np.ascontiguousarray(a.reshape(-1)),
                      np.ascontiguousarray(inst.b, dtype=np.float32).reshape(-1)]
        self.I, self.J, self.E = inst.I, inst.J, inst.E
        self.R = self.m * self.J  # rows of A: one dual entry each
        assert self._keep[3].shape[0] == self.m * self.E and self._keep[4].shape[0] == self.R
        self.weighted = bool(weighted)
        off, dst, c, a, b = self._keep
        self._h = self._lib.oracle_create_multi(self.I, self.J, self.m, _p(off), _p(dst), _p(c),
                                                _p(a), _p(b), int(weighted))
        if not self._h:
            raise MemoryError("oracle_create failed")
        self.box = bool(box)
        self._lib.oracle_set_box(self._h, int(box))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def row_scale(self) -> np.ndarray:
        D = np.empty(self.R, dtype=np.float64)
        self._lib.oracle_row_scale(self._h, _p(D))
        return D

    def norm2_sq(self, D=None) -> float:
        D = None if D is None else np.ascontiguousarray(D, dtype=np.float64)
        return float(self._lib.oracle_norm2_sq(self._h, _p(D)))

    def eval(self, mu, gamma: float, method: str = "sort", want_x: bool = False) -> Eval:
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        assert mu.shape == (self.R,)
        x = np.empty(self.E, dtype=np.float64) if want_x else None
        ax = np.empty(self.R, dtype=np.float64)
        grad = np.empty(self.R, dtype=np.float64)
        sc = np.empty(5, dtype=np.float64)
        rc = self._lib.oracle_eval(self._h, _p(mu), float(gamma), 0 if method == "sort" else 1,
                                   _p(x), _p(ax), _p(grad), _p(sc))
        if rc:
            raise RuntimeError(f"oracle_eval failed ({rc})")
        return Eval(float(sc[0]), float(sc[1]), float(sc[2]), float(sc[3]), float(sc[4]), grad,
                    ax, x)

    def solve(self, lam0=None, gamma0=0.1, gamma_final=1e-3, halve_every=25, max_step=10.0,
              init_step=1e-5, max_iters=2000, tol_gap=1e-4, tol_infeas=1e-4, check_every=10,
              row_normalize=True, restart=True, stop_on_tol=True, want_trace=False,
              restart_on_decrease=True):
        o = SolveOpts(gamma0, gamma_final, halve_every, max_step, init_step, max_iters, tol_gap,
                      tol_infeas, check_every, int(row_normalize), int(restart), int(stop_on_tol),
                      int(restart_on_decrease))
        lam = np.zeros(self.R) if lam0 is None else np.array(lam0, dtype=np.float64, copy=True)
        res = SolveResult()
        tr = np.zeros((max(max_iters, 1), TRACE_W)) if want_trace else None
        rc = self._lib.oracle_solve(self._h, ctypes.byref(o), _p(lam), ctypes.byref(res), _p(tr))
        if rc:
            raise RuntimeError(f"oracle_solve failed ({rc})")
        out = dict(iters=res.iters, converged=bool(res.converged), dual=res.dual,
                   primal_lin=res.primal_lin, reg=res.reg, infeas=res.infeas,
                   gap_rel=res.gap_rel, infeas_rel=res.infeas_rel, gamma=res.gamma, mu=lam,
                   restarts=res.restarts)
        if want_trace:
            out["trace"] = tr[: res.iters]
        return out
