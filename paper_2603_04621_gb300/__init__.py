"""Python binding of the dualip C ABI (include/dualip.h).

Argument marshalling only: every step of the dual evaluation and of the solve
runs in the CUDA kernels of ``libdualip.so`` (built in-tree by
:func:`paper_2603_04621_gb300.build.build`).  PyTorch provides device memory
and streams.  There is no CPU fallback: importing works without the library,
but every call raises if ``libdualip.so`` is missing or no GPU is present.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdualip.so")
_lib = None

DUALIP_OK, DUALIP_EINVAL, DUALIP_ENOMEM, DUALIP_ECUDA = 0, 1, 2, 3
DUALIP_ETIMEOUT, DUALIP_EBUSY, DUALIP_ENOTCONVERGED, DUALIP_EDEVICE = 4, 5, 6, 7
DUALIP_ECANCELED = 8
DUALIP_EDGE_F32, DUALIP_EDGE_BF16 = 0, 1
DUALIP_PROJ_SIMPLEX, DUALIP_PROJ_BOX = 0, 1
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EBUSY",
                6: "ENOTCONVERGED", 7: "EDEVICE", 8: "ECANCELED"}

# every entry point declared in include/dualip.h
EXPORTS = [
    "dualip_create", "dualip_destroy", "dualip_dual_grad", "dualip_dual_grad_async",
    "dualip_dual_grad_host", "dualip_get_primal", "dualip_check_device_status",
    "dualip_get_info", "dualip_solve_opts_default", "dualip_solve", "dualip_last_error",
    "dualip_profile_enable", "dualip_profile_collect", "dualip_dual_grad_noalloc",
    "dualip_batch_create", "dualip_batch_destroy", "dualip_batch_dual_grad",
    "dualip_batch_dual_grad_async", "dualip_batch_solve", "dualip_batch_autotune",
    "dualip_batch_set_tile_shape", "dualip_batch_get_info", "dualip_batch_profile_enable",
    "dualip_batch_profile_collect", "dualip_server_create", "dualip_server_submit",
    "dualip_server_poll", "dualip_server_wait", "dualip_server_get_stats",
    "dualip_server_destroy", "dualip_debug_abort_waits", "dualip_server_cancel",
    "dualip_solve_state_size", "dualip_solve_state_export", "dualip_solve_state_import",
]
DUALIP_REQ_QUEUED, DUALIP_REQ_RUNNING, DUALIP_REQ_DONE, DUALIP_REQ_FAILED = 0, 1, 2, 3


class DualipError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dualip {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class AutotuneResult(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int32), ("chosen", ctypes.c_int32),
                ("tile_edges", ctypes.c_int32 * 8), ("tile_sources", ctypes.c_int32 * 8),
                ("ms", ctypes.c_double * 8), ("degree_hist", ctypes.c_int64 * 32),
                ("lean80", ctypes.c_int32), ("pad", ctypes.c_int32), ("ms_lean80", ctypes.c_double)]

    def as_dict(self):
        n = self.n_candidates
        return dict(n_candidates=n, chosen=self.chosen, tile_edges=list(self.tile_edges[:n]),
                    tile_sources=list(self.tile_sources[:n]), ms=list(self.ms[:n]),
                    degree_hist=list(self.degree_hist), lean80=self.lean80,
                    ms_lean80=self.ms_lean80)


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32),
                ("check_every", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "queued", "running", "done", "failed",
                                              "resident_bytes", "peak_resident_bytes", "chunks",
                                              "slot_iterations")] + \
               [("busy_seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ProblemDesc(ctypes.Structure):
    _fields_ = [("num_sources", ctypes.c_int64), ("num_edges", ctypes.c_int64),
                ("num_dests", ctypes.c_int32), ("src_offsets", ctypes.c_void_p),
                ("dst", ctypes.c_void_p), ("c", ctypes.c_void_p), ("a", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("inputs_on_device", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("primal_scaling", ctypes.c_int32),
                ("projection", ctypes.c_int32), ("num_families", ctypes.c_int32)]


class Eval(ctypes.Structure):
    _fields_ = [("dual_obj", ctypes.c_double), ("primal_obj", ctypes.c_double),
                ("reg", ctypes.c_double), ("infeas_l2", ctypes.c_double),
                ("lambda_dot_grad", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveOpts(ctypes.Structure):
    _fields_ = [("gamma0", ctypes.c_double), ("gamma_final", ctypes.c_double),
                ("halve_every", ctypes.c_int32), ("max_step", ctypes.c_double),
                ("init_step", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("tol_gap", ctypes.c_double), ("tol_infeas", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("row_normalize", ctypes.c_int32),
                ("restart_on_gamma_change", ctypes.c_int32), ("stop_on_tol", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("restart_on_decrease", ctypes.c_int32),
                ("resume", ctypes.c_int32)]


class SolveResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("last", Eval),
                ("gap_rel", ctypes.c_double), ("infeas_rel", ctypes.c_double),
                ("gamma", ctypes.c_double)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("result", SolveResult),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("footprint_bytes", ctypes.c_int64),
                ("num_dests", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self):
        r = self.result
        return dict(state=self.state, status=self.status, t_submit=self.t_submit,
                    t_admit=self.t_admit, t_done=self.t_done,
                    footprint_bytes=self.footprint_bytes, iters=r.iters,
                    converged=bool(r.converged), gap_rel=r.gap_rel, infeas_rel=r.infeas_rel,
                    gamma=r.gamma, **r.last.as_dict())


def lib() -> ctypes.CDLL:
    """Load libdualip.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2603_04621_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        st = ctypes.c_int
        L.dualip_create.argtypes = [ctypes.POINTER(ProblemDesc), vp, ctypes.POINTER(vp)]
        L.dualip_create.restype = st
        L.dualip_destroy.argtypes = [vp]
        L.dualip_destroy.restype = None
        L.dualip_dual_grad.argtypes = [vp, vp, dbl, vp, ctypes.POINTER(Eval), vp]
        L.dualip_dual_grad.restype = st
        L.dualip_dual_grad_async.argtypes = [vp, vp, dbl, vp, vp, vp]
        L.dualip_dual_grad_async.restype = st
        L.dualip_dual_grad_host.argtypes = [vp, vp, dbl, vp, ctypes.POINTER(Eval), vp]
        L.dualip_dual_grad_host.restype = st
        L.dualip_get_primal.argtypes = [vp, vp, dbl, vp, vp]
        L.dualip_get_primal.restype = st
        L.dualip_check_device_status.argtypes = [vp, vp]
        L.dualip_check_device_status.restype = st
        L.dualip_get_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                      ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.dualip_get_info.restype = st
        L.dualip_solve_opts_default.argtypes = [ctypes.POINTER(SolveOpts)]
        L.dualip_solve_opts_default.restype = None
        L.dualip_solve.argtypes = [vp, ctypes.POINTER(SolveOpts), vp, ctypes.POINTER(SolveResult),
                                   vp, vp]
        L.dualip_solve.restype = st
        L.dualip_profile_enable.argtypes = [vp, i32]
        L.dualip_profile_enable.restype = st
        pd = ctypes.POINTER(dbl)
        L.dualip_profile_collect.argtypes = [vp, pd, pd, pd, ctypes.POINTER(i32)]
        L.dualip_profile_collect.restype = st
        L.dualip_dual_grad_noalloc.argtypes = [i64, i32, vp, vp, vp, vp, vp, i32, vp, dbl, vp,
                                               vp, vp]
        L.dualip_dual_grad_noalloc.restype = st
        L.dualip_batch_create.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.dualip_batch_create.restype = st
        L.dualip_batch_destroy.argtypes = [vp]
        L.dualip_batch_destroy.restype = None
        L.dualip_batch_dual_grad.argtypes = [vp, vp, ctypes.POINTER(dbl), vp,
                                             ctypes.POINTER(Eval), vp]
        L.dualip_batch_dual_grad.restype = st
        L.dualip_batch_dual_grad_async.argtypes = [vp, vp, ctypes.POINTER(dbl), vp, vp, vp]
        L.dualip_batch_dual_grad_async.restype = st
        L.dualip_batch_solve.argtypes = [vp, ctypes.POINTER(SolveOpts), i32, vp,
                                         ctypes.POINTER(SolveResult), vp]
        L.dualip_batch_solve.restype = st
        L.dualip_batch_autotune.argtypes = [vp, ctypes.POINTER(AutotuneResult), vp]
        L.dualip_batch_autotune.restype = st
        L.dualip_batch_set_tile_shape.argtypes = [vp, i32, i32]
        L.dualip_batch_set_tile_shape.restype = st
        L.dualip_batch_get_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                            ctypes.POINTER(i64), ctypes.POINTER(i64),
                                            ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.dualip_batch_get_info.restype = st
        L.dualip_batch_profile_enable.argtypes = [vp, i32]
        L.dualip_batch_profile_enable.restype = st
        L.dualip_batch_profile_collect.argtypes = [vp, pd, pd, pd, ctypes.POINTER(i32)]
        L.dualip_batch_profile_collect.restype = st
        L.dualip_server_create.argtypes = [ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
        L.dualip_server_create.restype = st
        L.dualip_server_submit.argtypes = [vp, ctypes.POINTER(ProblemDesc),
                                           ctypes.POINTER(SolveOpts), ctypes.POINTER(i64)]
        L.dualip_server_submit.restype = st
        L.dualip_server_poll.argtypes = [vp, i64, ctypes.POINTER(RequestInfo), vp]
        L.dualip_server_poll.restype = st
        L.dualip_server_wait.argtypes = [vp, i64, dbl, ctypes.POINTER(RequestInfo), vp]
        L.dualip_server_wait.restype = st
        L.dualip_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.dualip_server_get_stats.restype = st
        L.dualip_server_destroy.argtypes = [vp]
        L.dualip_server_destroy.restype = None
        L.dualip_server_cancel.argtypes = [vp, i64]
        L.dualip_server_cancel.restype = st
        L.dualip_debug_abort_waits.argtypes = [vp, vp]
        L.dualip_debug_abort_waits.restype = st
        L.dualip_solve_state_size.argtypes = [vp, ctypes.POINTER(i64)]
        L.dualip_solve_state_size.restype = st
        L.dualip_solve_state_export.argtypes = [vp, vp, i64, vp]
        L.dualip_solve_state_export.restype = st
        L.dualip_solve_state_import.argtypes = [vp, vp, i64, vp]
        L.dualip_solve_state_import.restype = st
        L.dualip_last_error.argtypes = []
        L.dualip_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int, ok=(DUALIP_OK,)) -> int:
    if status not in ok:
        raise DualipError(status, lib().dualip_last_error().decode())
    return status


def _stream(stream=None) -> int:
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _ptr(x) -> int:
    """Address of a contiguous numpy array or torch tensor."""
    if x is None:
        return 0
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return int(x.ctypes.data)
    assert x.is_contiguous()
    return int(x.data_ptr())


# ------------------------------------------------------------ C ABI, 1:1 ----
def dualip_create(desc: ProblemDesc, stream: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().dualip_create(ctypes.byref(desc), stream, ctypes.byref(h)))
    return int(h.value)


def dualip_destroy(h: int) -> None:
    if h:
        lib().dualip_destroy(h)


def dualip_dual_grad(h: int, lam_ptr: int, gamma: float, grad_ptr: int, stream: int,
                     want_eval: bool = True):
    ev = Eval()
    _check(lib().dualip_dual_grad(h, lam_ptr, gamma, grad_ptr,
                                  ctypes.byref(ev) if want_eval else None, stream))
    return ev if want_eval else None


def dualip_dual_grad_async(h: int, lam_ptr: int, gamma: float, grad_ptr: int, out_ptr: int,
                           stream: int) -> None:
    _check(lib().dualip_dual_grad_async(h, lam_ptr, gamma, grad_ptr, out_ptr, stream))


def dualip_dual_grad_host(h: int, lam_host_ptr: int, gamma: float, grad_host_ptr: int,
                          stream: int) -> Eval:
    ev = Eval()
    _check(lib().dualip_dual_grad_host(h, lam_host_ptr, gamma, grad_host_ptr, ctypes.byref(ev),
                                       stream))
    return ev


def dualip_get_primal(h: int, lam_ptr: int, gamma: float, x_ptr: int, stream: int) -> None:
    _check(lib().dualip_get_primal(h, lam_ptr, gamma, x_ptr, stream))


def dualip_check_device_status(h: int, stream: int) -> None:
    _check(lib().dualip_check_device_status(h, stream))


def dualip_get_info(h: int) -> dict:
    I, J, E, T = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().dualip_get_info(h, ctypes.byref(I), ctypes.byref(J), ctypes.byref(E),
                                 ctypes.byref(T)))
    return dict(I=I.value, J=J.value, E=E.value, tiles=T.value)


def dualip_profile_enable(h: int, max_evals: int) -> None:
    _check(lib().dualip_profile_enable(h, int(max_evals)))


def dualip_profile_collect(h: int) -> dict:
    a, b, c, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(lib().dualip_profile_collect(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                        ctypes.byref(n)))
    return dict(ms_prologue=a.value, ms_pass=b.value, ms_epilogue=c.value, count=n.value)


def dualip_dual_grad_noalloc(I: int, J: int, off_ptr: int, dst_ptr: int, c_ptr: int, a_ptr: int,
                             b_ptr: int, primal_scaling: int, lam_ptr: int, gamma: float,
                             grad_ptr: int, out_ptr: int, stream: int) -> None:
    """The allocation-free evaluation (all pointers are device pointers)."""
    _check(lib().dualip_dual_grad_noalloc(I, J, off_ptr, dst_ptr, c_ptr, a_ptr, b_ptr,
                                          int(primal_scaling), lam_ptr, gamma, grad_ptr,
                                          out_ptr, stream))


def dualip_solve_opts_default() -> SolveOpts:
    o = SolveOpts()
    lib().dualip_solve_opts_default(ctypes.byref(o))
    return o


def dualip_solve(h: int, opts: SolveOpts, lam_ptr: int, trace_ptr: int, stream: int):
    r = SolveResult()
    st = lib().dualip_solve(h, ctypes.byref(opts), lam_ptr, ctypes.byref(r), trace_ptr, stream)
    _check(st, ok=(DUALIP_OK, DUALIP_ENOTCONVERGED))
    return r


def dualip_solve_state_size(h: int) -> int:
    n = ctypes.c_int64()
    _check(lib().dualip_solve_state_size(h, ctypes.byref(n)))
    return n.value


def dualip_solve_state_export(h: int, buf_ptr: int, nbytes: int, stream: int) -> None:
    _check(lib().dualip_solve_state_export(h, buf_ptr, nbytes, stream))


def dualip_solve_state_import(h: int, buf_ptr: int, nbytes: int, stream: int) -> None:
    _check(lib().dualip_solve_state_import(h, buf_ptr, nbytes, stream))


def dualip_batch_create(handles) -> int:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    out = ctypes.c_void_p()
    _check(lib().dualip_batch_create(len(handles), arr, ctypes.byref(out)))
    return out.value


def dualip_batch_destroy(b: int) -> None:
    lib().dualip_batch_destroy(b)


def _doubles(xs):
    return (ctypes.c_double * len(xs))(*[float(x) for x in xs])


def dualip_batch_dual_grad(b: int, lam_ptr: int, gammas, grad_ptr: int, stream: int):
    out = (Eval * len(gammas))()
    _check(lib().dualip_batch_dual_grad(b, lam_ptr, _doubles(gammas), grad_ptr, out, stream))
    return [e.as_dict() for e in out]


def dualip_batch_dual_grad_async(b: int, lam_ptr: int, gammas, grad_ptr: int, out_dev_ptr: int,
                                 stream: int) -> None:
    _check(lib().dualip_batch_dual_grad_async(b, lam_ptr, _doubles(gammas), grad_ptr,
                                              out_dev_ptr, stream))


def dualip_batch_solve(b: int, opts, lam_ptr: int, n: int, stream: int):
    opts = list(opts) if isinstance(opts, (list, tuple)) else [opts]
    oa = (SolveOpts * len(opts))(*opts)
    res = (SolveResult * n)()
    _check(lib().dualip_batch_solve(b, oa, len(opts), lam_ptr, res, stream),
           ok=(DUALIP_OK, DUALIP_ENOTCONVERGED))
    return list(res)


def dualip_batch_autotune(b: int, stream: int) -> dict:
    r = AutotuneResult()
    _check(lib().dualip_batch_autotune(b, ctypes.byref(r), stream))
    return r.as_dict()


def dualip_batch_set_tile_shape(b: int, edges: int, sources: int) -> None:
    _check(lib().dualip_batch_set_tile_shape(b, edges, sources))


def dualip_batch_get_info(b: int) -> dict:
    n, te, ts = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    J, E, T = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().dualip_batch_get_info(b, ctypes.byref(n), ctypes.byref(J), ctypes.byref(E),
                                       ctypes.byref(T), ctypes.byref(te), ctypes.byref(ts)))
    return dict(n=n.value, J=J.value, E=E.value, ntiles=T.value, tile_edges=te.value,
                tile_sources=ts.value)


def dualip_batch_profile_enable(b: int, max_evals: int) -> None:
    _check(lib().dualip_batch_profile_enable(b, max_evals))


def dualip_batch_profile_collect(b: int) -> dict:
    t = [ctypes.c_double() for _ in range(3)]
    n = ctypes.c_int32()
    _check(lib().dualip_batch_profile_collect(b, *[ctypes.byref(x) for x in t], ctypes.byref(n)))
    return dict(ms_prologue=t[0].value, ms_pass=t[1].value, ms_epilogue=t[2].value,
                count=n.value)


def dualip_server_create(budget_bytes: int, max_slots: int, check_every: int = 10) -> int:
    o = ServerOpts(int(budget_bytes), int(max_slots), int(check_every))
    out = ctypes.c_void_p()
    _check(lib().dualip_server_create(ctypes.byref(o), ctypes.byref(out)))
    return out.value


def dualip_server_submit(srv: int, desc: "ProblemDesc", opts) -> int:
    t = ctypes.c_int64()
    _check(lib().dualip_server_submit(srv, ctypes.byref(desc),
                                      ctypes.byref(opts) if opts is not None else None,
                                      ctypes.byref(t)))
    return t.value


def dualip_server_poll(srv: int, ticket: int, lam_ptr: int = 0) -> dict:
    info = RequestInfo()
    _check(lib().dualip_server_poll(srv, ticket, ctypes.byref(info), lam_ptr or None))
    return info.as_dict()


def dualip_server_wait(srv: int, ticket: int, timeout_s: float, lam_ptr: int = 0) -> dict:
    info = RequestInfo()
    _check(lib().dualip_server_wait(srv, ticket, float(timeout_s), ctypes.byref(info),
                                    lam_ptr or None))
    return info.as_dict()


def dualip_server_get_stats(srv: int) -> dict:
    st = ServerStats()
    _check(lib().dualip_server_get_stats(srv, ctypes.byref(st)))
    return st.as_dict()


def dualip_server_cancel(srv: int, ticket: int) -> None:
    _check(lib().dualip_server_cancel(srv, ticket))


def dualip_server_destroy(srv: int) -> None:
    lib().dualip_server_destroy(srv)


def dualip_debug_abort_waits(h: int, stream: int) -> None:
    _check(lib().dualip_debug_abort_waits(h, stream))


# ------------------------------------------------- convenience (marshalling) ----
class Problem:
    """Owns one dualip handle built from host (numpy) or device (torch) arrays.

    ``off`` int64 [I+1], ``dst`` int32 [E], ``c``/``a`` float32 [E], ``b`` float32 [J].
    """

    def __init__(self, off, dst, c, a, b, J: int, storage: str = "f32",
                 primal_scaling: bool = False, projection: str = "simplex", stream=None):
        import torch

        on_dev = isinstance(off, torch.Tensor) and off.is_cuda
        if not on_dev:
            off = np.ascontiguousarray(off, dtype=np.int64)
            dst = np.ascontiguousarray(dst, dtype=np.int32)
            c = np.ascontiguousarray(c, dtype=np.float32)
            a = np.ascontiguousarray(a, dtype=np.float32)
            b = np.ascontiguousarray(b, dtype=np.float32)
        # a: [E] (one constraint family) or [m, E] (m families, family-major);
        # the dual then has m J entries (row k J + j), and self.J counts them
        m = 1 if a.ndim == 1 else int(a.shape[0])
        self._keep = (off, dst, c, a, b)
        I = int(off.shape[0]) - 1
        E = int(dst.shape[0])
        self.I, self.E, self.m, self.num_dests = I, E, m, int(J)
        self.J = m * int(J)
        self.storage = storage
        d = ProblemDesc(I, E, int(J), _ptr(off), _ptr(dst), _ptr(c), _ptr(a), _ptr(b),
                        1 if on_dev else 0,
                        DUALIP_EDGE_BF16 if storage == "bf16" else DUALIP_EDGE_F32,
                        1 if primal_scaling else 0,
                        DUALIP_PROJ_BOX if projection == "box" else DUALIP_PROJ_SIMPLEX, m)
        self.h = dualip_create(d, _stream(stream))
        self._keep = None
        self.device = torch.device("cuda", torch.cuda.current_device())

    @classmethod
    def from_instance(cls, inst, **kw) -> "Problem":
        return cls(inst.off, inst.dst, inst.c, inst.a, inst.b, inst.J, **kw)

    def close(self):
        if getattr(self, "h", 0):
            dualip_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return dualip_get_info(self.h)

    def _dev_vec(self, v, n):
        import torch

        if isinstance(v, torch.Tensor):
            assert v.is_cuda and v.dtype == torch.float32 and v.numel() == n
            return v.contiguous()
        return torch.as_tensor(np.asarray(v, dtype=np.float32), device=self.device)

    def dual_grad(self, lam, gamma: float, grad=None, stream=None):
        """grad = A x*(lam) - b on the device and the FP64 scalars (dict)."""
        import torch

        lam = self._dev_vec(lam, self.J)
        if grad is None:
            grad = torch.empty(self.J, dtype=torch.float32, device=self.device)
        ev = dualip_dual_grad(self.h, _ptr(lam), float(gamma), _ptr(grad), _stream(stream))
        return grad, ev.as_dict()

    def primal(self, lam, gamma: float, stream=None):
        import torch

        lam = self._dev_vec(lam, self.J)
        x = torch.empty(self.E, dtype=torch.float32, device=self.device)
        dualip_get_primal(self.h, _ptr(lam), float(gamma), _ptr(x), _stream(stream))
        return x

    def solve(self, lam0=None, trace: bool = False, stream=None, **opts):
        """Run dualip_solve; returns (lam tensor, result dict[, trace ndarray])."""
        import torch

        o = dualip_solve_opts_default()
        for k, v in opts.items():
            if k == "restart":
                k = "restart_on_gamma_change"
            setattr(o, k, v)
        lam = (torch.zeros(self.J, dtype=torch.float32, device=self.device) if lam0 is None
               else self._dev_vec(lam0, self.J).clone())
        tr = torch.zeros((max(o.max_iters, 1), 8), dtype=torch.float64, device=self.device) \
            if trace else None
        r = dualip_solve(self.h, o, _ptr(lam), _ptr(tr), _stream(stream))
        res = dict(iters=r.iters, converged=bool(r.converged), gap_rel=r.gap_rel,
                   infeas_rel=r.infeas_rel, gamma=r.gamma, **r.last.as_dict())
        if trace:
            return lam, res, tr[: r.iters].cpu().numpy()
        return lam, res

    def export_state(self, stream=None) -> np.ndarray:
        """The handle's saved ascent (dualip_solve_state_export) as a byte array."""
        buf = np.empty(dualip_solve_state_size(self.h), dtype=np.uint8)
        dualip_solve_state_export(self.h, _ptr(buf), buf.nbytes, _stream(stream))
        return buf

    def import_state(self, buf: np.ndarray, stream=None) -> None:
        """Load a saved ascent; the next solve(resume=1) continues from it."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        dualip_solve_state_import(self.h, _ptr(buf), buf.nbytes, _stream(stream))


class Batch:
    """A dualip batch over Problem objects (which must outlive it).  Joint
    vectors hold the problems' destination vectors back to back."""

    def __init__(self, problems):
        import torch

        self.problems = list(problems)
        self.h = dualip_batch_create([p.h for p in self.problems])
        self.Js = [p.J for p in self.problems]
        self.joff = np.concatenate([[0], np.cumsum(self.Js)]).astype(np.int64)
        self.device = torch.device("cuda", torch.cuda.current_device())

    @property
    def n(self) -> int:
        return len(self.problems)

    def close(self):
        if getattr(self, "h", 0):
            dualip_batch_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def split(self, v):
        return [v[self.joff[k]:self.joff[k + 1]] for k in range(self.n)]

    def dual_grad(self, lam, gammas, stream=None):
        """lam: joint torch vector; returns (joint grad tensor, list of scalar dicts)."""
        import torch

        assert lam.is_cuda and lam.dtype == torch.float32 and lam.numel() == int(self.joff[-1])
        grad = torch.empty_like(lam)
        ev = dualip_batch_dual_grad(self.h, _ptr(lam.contiguous()), gammas, _ptr(grad),
                                    _stream(stream))
        return grad, ev

    def solve(self, lam0=None, opts=None, stream=None, **kw):
        """Per-problem ascent; opts: a list of per-problem dicts or one dict (kw)."""
        import torch

        def mk(d):
            o = dualip_solve_opts_default()
            for k, v in d.items():
                setattr(o, "restart_on_gamma_change" if k == "restart" else k, v)
            return o

        ol = [mk(d) for d in opts] if opts is not None else [mk(kw)]
        lam = (torch.zeros(int(self.joff[-1]), dtype=torch.float32, device=self.device)
               if lam0 is None else lam0.clone())
        res = dualip_batch_solve(self.h, ol, _ptr(lam), self.n, _stream(stream))
        out = [dict(iters=r.iters, converged=bool(r.converged), gap_rel=r.gap_rel,
                    infeas_rel=r.infeas_rel, gamma=r.gamma, **r.last.as_dict()) for r in res]
        return lam, out

    def autotune(self, stream=None) -> dict:
        return dualip_batch_autotune(self.h, _stream(stream))

    def set_tile_shape(self, edges: int, sources: int) -> None:
        dualip_batch_set_tile_shape(self.h, edges, sources)

    def info(self) -> dict:
        return dualip_batch_get_info(self.h)


class Server:
    """The serving loop.  submit() keeps the request's host arrays alive until
    it has been admitted; wait() returns (info dict, lambda ndarray or None)."""

    def __init__(self, budget_bytes: int, max_slots: int = 64, check_every: int = 10):
        self.h = dualip_server_create(budget_bytes, max_slots, check_every)
        self._keep = {}
        self._J = {}

    def submit(self, inst, storage: str = "f32", primal_scaling: bool = False, **opts) -> int:
        arrs = (np.ascontiguousarray(inst.off, dtype=np.int64),
                np.ascontiguousarray(inst.dst, dtype=np.int32),
                np.ascontiguousarray(inst.c, dtype=np.float32),
                np.ascontiguousarray(inst.a, dtype=np.float32),
                np.ascontiguousarray(inst.b, dtype=np.float32))
        d = ProblemDesc(inst.I, inst.E, inst.J, *[a.ctypes.data for a in arrs], 0,
                        DUALIP_EDGE_BF16 if storage == "bf16" else DUALIP_EDGE_F32,
                        1 if primal_scaling else 0)
        o = dualip_solve_opts_default()
        for k, v in opts.items():
            setattr(o, "restart_on_gamma_change" if k == "restart" else k, v)
        t = dualip_server_submit(self.h, d, o)
        self._keep[t] = arrs
        self._J[t] = inst.J
        return t

    def poll(self, ticket: int) -> dict:
        info = dualip_server_poll(self.h, ticket)
        if info["state"] != DUALIP_REQ_QUEUED:
            self._keep.pop(ticket, None)
        return info

    def wait(self, ticket: int, timeout_s: float = 600.0):
        lam = np.empty(self._J[ticket], dtype=np.float32)
        info = dualip_server_wait(self.h, ticket, timeout_s, lam.ctypes.data)
        if info["state"] != DUALIP_REQ_QUEUED:  # the build has copied the arrays
            self._keep.pop(ticket, None)
        return info, (lam if info["state"] == DUALIP_REQ_DONE else None)

    def stats(self) -> dict:
        return dualip_server_get_stats(self.h)

    def cancel(self, ticket: int) -> None:
        dualip_server_cancel(self.h, ticket)

    def close(self):
        if getattr(self, "h", 0):
            dualip_server_destroy(self.h)
            self.h = 0
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
