"""Python binding of the GB300 batched nonlinear solver (``include/nls.h``).

The functions named ``nls_*`` are one-to-one ctypes bindings of the C ABI:
they marshal arguments and nothing else; every step of a solve runs in the
CUDA kernels of ``_lib/libnls.so``.  ``Solver`` and ``solve`` are small
conveniences over them for torch tensors (device memory and the current
stream come from PyTorch).

There is no CPU fallback: if the CUDA library has not been built, or no GPU
is present, calls raise instead of computing anything elsewhere.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import inputs  # noqa: F401  (seeded workload generator)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libnls.so")

# nls_family
NLS_CUBIC, NLS_BRATU, NLS_SQUARE, NLS_ROSENBROCK = 0, 1, 2, 3
# nls_alg and flags
NLS_NEWTON, NLS_NEWTON_BACKTRACK, NLS_TRUST_DOGLEG, NLS_POLYALG = 0, 1, 2, 3
NLS_POTRA_PTAK, NLS_HALLEY, NLS_BROYDEN, NLS_MOD_BROYDEN = 4, 5, 6, 7
NLS_ALG_MASK = 0xFF
NLS_MIXED = 1 << 8
NLS_ANALYTIC_JAC = 1 << 9
NLS_TILE_THREAD = 1 << 10
NLS_TILE_WARP = 1 << 11
NLS_TILE_CTA = 1 << 12
NLS_TR_NOCEDAL_WRIGHT = 1 << 13
NLS_REFINE = 1 << 14
# nls_inst_status
(NLS_SUCCESS, NLS_MAXITERS, NLS_SINGULAR, NLS_NONFINITE, NLS_LS_FAILED, NLS_TR_STALLED,
 NLS_ABORTED) = range(7)
# nls_err
NLS_OK, NLS_E_INVALID, NLS_E_CUDA, NLS_E_NOMEM = 0, -1, -2, -3
NLS_E_UNSUPPORTED, NLS_E_TIMEOUT, NLS_E_BUSY, NLS_E_NOTFOUND = -4, -5, -6, -7
# nls_option
NLS_OPT_PERSISTENT, NLS_OPT_REFILL_BELOW, NLS_OPT_CTAS_PER_SM, NLS_OPT_GRAPH = 1, 2, 3, 4
NLS_OPT_DEADLINE_US = 5

EXPORTED = ("nls_batch_create", "nls_solve", "nls_flush", "nls_status", "nls_solve_host",
            "nls_solve_host_async",
            "nls_batch_destroy", "nls_last_error", "nls_launch_count", "nls_set_option",
            "nls_solve_noalloc", "nls_autotune", "nls_tune_save", "nls_tune_load",
            "nls_server_create", "nls_server_submit", "nls_server_wait", "nls_server_wait_timed",
            "nls_server_now",
            "nls_server_stats", "nls_server_destroy", "nls_tune_lookup", "nls_adjoint")
NLS_NOALLOC_MAX_GROUPS = 64


class NlsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"nls error {code}: {msg}")
        self.code = code


class nls_outputs(ctypes.Structure):
    _fields_ = [("status", ctypes.c_void_p), ("iters", ctypes.c_void_p),
                ("resid_inf", ctypes.c_void_p), ("nfev", ctypes.c_void_p),
                ("ngrad", ctypes.c_void_p)]


class nls_server_timing(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double),
                ("h2d_ms", ctypes.c_float), ("solve_ms", ctypes.c_float),
                ("d2h_ms", ctypes.c_float), ("wave_requests", ctypes.c_int)]


class nls_group(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("n", ctypes.c_int), ("params", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("batch", ctypes.c_int64), ("out", nls_outputs)]


_lock = threading.Lock()
_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load ``libnls.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library {p} is missing: build it with "
                               "paper_2403_16341_gb300.build.build()")
        lib = ctypes.CDLL(p)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        out_p = ctypes.POINTER(nls_outputs)
        sig = {
            "nls_batch_create": ([ctypes.POINTER(vp), i32, vp, ctypes.c_size_t], i32),
            "nls_solve": ([vp, i32, vp, vp, i32, i64, i32, dbl, i32, out_p,
                           ctypes.POINTER(i64)], i32),
            "nls_flush": ([vp], i32),
            "nls_status": ([vp, i64, ctypes.POINTER(i64), i32], i32),
            "nls_solve_host": ([vp, i32, vp, vp, i32, i64, i32, dbl, i32, out_p,
                                ctypes.POINTER(i64)], i32),
            "nls_solve_host_async": ([vp, i32, vp, vp, i32, i64, i32, dbl, i32, out_p,
                                      ctypes.POINTER(i64)], i32),
            "nls_batch_destroy": ([vp], i32),
            "nls_last_error": ([vp], ctypes.c_char_p),
            "nls_launch_count": ([vp], i64),
            "nls_set_option": ([vp, i32, i64], i32),
            "nls_solve_noalloc": ([vp, ctypes.POINTER(nls_group), i32, i32, dbl, i32,
                                   ctypes.POINTER(i64)], i32),
            "nls_autotune": ([vp, i32, vp, vp, i32, i64, i32, dbl, i32,
                              ctypes.POINTER(ctypes.c_int)], i32),
            "nls_tune_save": ([vp, ctypes.c_char_p], i32),
            "nls_adjoint": ([vp, i32, vp, vp, i32, i64, vp, vp, vp], i32),
            "nls_tune_lookup": ([vp, i32, i32, i32, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(dbl)], i32),
            "nls_tune_load": ([vp, ctypes.c_char_p], i32),
            "nls_server_create": ([ctypes.POINTER(vp), i32, ctypes.c_size_t, i32], i32),
            "nls_server_submit": ([vp, i32, vp, vp, i32, i64, i32, dbl, i32, out_p,
                                   ctypes.POINTER(i64)], i32),
            "nls_server_wait": ([vp, i64, ctypes.POINTER(i64), ctypes.POINTER(dbl),
                                 ctypes.POINTER(dbl), i32], i32),
            "nls_server_wait_timed": ([vp, i64, ctypes.POINTER(i64),
                                       ctypes.POINTER(nls_server_timing), i32], i32),
            "nls_server_now": ([vp], dbl),
            "nls_server_stats": ([vp, ctypes.POINTER(i64), i32], i32),
            "nls_server_destroy": ([vp], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


# ------------------------------------------------------------- raw C ABI

def nls_batch_create(device: int = 0, stream: int = 0, mem_cap_bytes: int = 0) -> int:
    lib = load_library()
    h = ctypes.c_void_p()
    rc = lib.nls_batch_create(ctypes.byref(h), device, ctypes.c_void_p(stream or None),
                              mem_cap_bytes)
    if rc:
        raise NlsError(rc, lib.nls_last_error(None).decode())
    return h.value


def _check(h, rc: int) -> int:
    if rc:
        raise NlsError(rc, load_library().nls_last_error(h).decode())
    return rc


def _outs(status=0, iters=0, resid=0, nfev=0, ngrad=0):
    return nls_outputs(status or None, iters or None, resid or None, nfev or None, ngrad or None)


def nls_solve(h, family, params, u, n, batch, alg, abstol, maxiters, status=0, iters=0,
              resid_inf=0, nfev=0, ngrad=0) -> int:
    """Enqueue a solve on raw device addresses; returns the request id."""
    req = ctypes.c_int64()
    out = _outs(status, iters, resid_inf, nfev, ngrad)
    _check(h, load_library().nls_solve(h, family, params or None, u or None, n, batch, alg,
                                       abstol, maxiters, ctypes.byref(out), ctypes.byref(req)))
    return req.value


def nls_flush(h) -> None:
    _check(h, load_library().nls_flush(h))


def nls_status(h, req: int, timeout_ms: int = -1):
    """Returns the number of solved instances, or None on NLS_E_TIMEOUT."""
    s = ctypes.c_int64(-1)
    rc = load_library().nls_status(h, req, ctypes.byref(s), timeout_ms)
    if rc == NLS_E_TIMEOUT:
        return None
    _check(h, rc)
    return s.value


def nls_solve_host(h, family, params, u, n, batch, alg, abstol, maxiters, status=0, iters=0,
                   resid_inf=0, nfev=0, ngrad=0) -> int:
    """Synchronous solve on raw HOST addresses; returns the solved count."""
    s = ctypes.c_int64(-1)
    out = _outs(status, iters, resid_inf, nfev, ngrad)
    _check(h, load_library().nls_solve_host(h, family, params or None, u or None, n, batch, alg,
                                            abstol, maxiters, ctypes.byref(out), ctypes.byref(s)))
    return s.value


def nls_solve_host_async(h, family, params, u, n, batch, alg, abstol, maxiters, status=0, iters=0,
                         resid_inf=0, nfev=0, ngrad=0) -> int:
    """Enqueue a solve on raw HOST addresses; returns the request id for
    nls_status (the host buffers must stay untouched until then)."""
    req = ctypes.c_int64()
    out = _outs(status, iters, resid_inf, nfev, ngrad)
    _check(h, load_library().nls_solve_host_async(h, family, params or None, u or None, n, batch,
                                                  alg, abstol, maxiters, ctypes.byref(out),
                                                  ctypes.byref(req)))
    return req.value


def nls_batch_destroy(h) -> None:
    _check(h, load_library().nls_batch_destroy(h))


def nls_last_error(h) -> str:
    return load_library().nls_last_error(h).decode()


def nls_launch_count(h) -> int:
    return load_library().nls_launch_count(h)


def nls_set_option(h, option: int, value: int) -> None:
    _check(h, load_library().nls_set_option(h, option, value))


def nls_solve_noalloc(stream, groups, alg, abstol, maxiters, want_solved=True):
    """Allocation-free solve of up to NLS_NOALLOC_MAX_GROUPS groups.

    ``groups``: sequence of (family, n, params_ptr, u_ptr, batch,
    (status_ptr, iters_ptr, resid_ptr, nfev_ptr)) with raw DEVICE addresses
    (0 = none).  Returns the per-group solved counts (waits for the stream),
    or None when ``want_solved`` is False (returns after enqueueing)."""
    arr = (nls_group * max(len(groups), 1))()
    for i, (fam, n, p, u, b, outs) in enumerate(groups):
        arr[i] = nls_group(fam, n, p or None, u or None, b, _outs(*outs))
    solved = (ctypes.c_int64 * max(len(groups), 1))()
    lib = load_library()
    rc = lib.nls_solve_noalloc(ctypes.c_void_p(stream or None), arr, len(groups), alg, abstol,
                               maxiters, solved if want_solved else None)
    if rc:
        raise NlsError(rc, lib.nls_last_error(None).decode())
    return list(solved[:len(groups)]) if want_solved else None


def nls_autotune(h, family, params, u, n, batch, alg, abstol, maxiters) -> int:
    """Time the tilings that can hold n on this batch; returns the chosen NLS_TILE_* flag."""
    chosen = ctypes.c_int(0)
    _check(h, load_library().nls_autotune(h, family, params or None, u or None, n, batch, alg,
                                          abstol, maxiters, ctypes.byref(chosen)))
    return chosen.value


def nls_adjoint(h, family, params, u, n, batch, w, grad, status=0) -> None:
    """dL/dtheta at the roots for cotangents w (raw DEVICE addresses)."""
    _check(h, load_library().nls_adjoint(h, family, params or None, u or None, n, batch,
                                         w or None, grad or None, status or None))


def nls_tune_lookup(h, family, n, alg) -> dict:
    """The tuned entry: tiles, lanes, refill (-2 = one block per chunk), rate."""
    t, l, r, q = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(h, load_library().nls_tune_lookup(h, family, n, alg, ctypes.byref(t), ctypes.byref(l),
                                             ctypes.byref(r), ctypes.byref(q)))
    return {"tiles": t.value, "lanes": l.value, "refill": r.value, "rate": q.value}


def nls_tune_save(h, path: str) -> None:
    _check(h, load_library().nls_tune_save(h, path.encode()))


def nls_tune_load(h, path: str) -> None:
    _check(h, load_library().nls_tune_load(h, path.encode()))


def _gcheck(rc: int) -> None:
    if rc:
        raise NlsError(rc, load_library().nls_last_error(None).decode())


def nls_server_create(device: int = 0, mem_budget_bytes: int = 0, streams: int = 4):
    s = ctypes.c_void_p()
    _gcheck(load_library().nls_server_create(ctypes.byref(s), device, mem_budget_bytes, streams))
    return s.value


def nls_server_submit(s, family, params, u, n, batch, alg, abstol, maxiters, status=0, iters=0,
                      resid_inf=0, nfev=0, ngrad=0) -> int:
    """Queue a request on raw HOST addresses; returns its ticket."""
    t = ctypes.c_int64()
    out = _outs(status, iters, resid_inf, nfev, ngrad)
    _gcheck(load_library().nls_server_submit(s, family, params or None, u or None, n, batch, alg,
                                             abstol, maxiters, ctypes.byref(out), ctypes.byref(t)))
    return t.value


def nls_server_wait(s, ticket: int, timeout_ms: int = -1):
    """Returns (solved, t_submit, t_done) or None on NLS_E_TIMEOUT."""
    sv, ts, td = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    rc = load_library().nls_server_wait(s, ticket, ctypes.byref(sv), ctypes.byref(ts),
                                        ctypes.byref(td), timeout_ms)
    if rc == NLS_E_TIMEOUT:
        return None
    _gcheck(rc)
    return sv.value, ts.value, td.value


def nls_server_wait_timed(s, ticket: int, timeout_ms: int = -1):
    """Returns (solved, timing dict) or None on NLS_E_TIMEOUT."""
    sv, tm = ctypes.c_int64(), nls_server_timing()
    rc = load_library().nls_server_wait_timed(s, ticket, ctypes.byref(sv), ctypes.byref(tm),
                                              timeout_ms)
    if rc == NLS_E_TIMEOUT:
        return None
    _gcheck(rc)
    return sv.value, {f: getattr(tm, f) for f, _ in nls_server_timing._fields_}


def nls_server_now(s) -> float:
    return load_library().nls_server_now(s)


SERVER_COUNTERS = ("admitted", "completed", "solved", "max_queue", "max_inflight", "waves",
                   "queued", "inflight", "arena_bytes", "largest_free")


def nls_server_stats(s) -> dict:
    c = (ctypes.c_int64 * len(SERVER_COUNTERS))()
    _gcheck(load_library().nls_server_stats(s, c, len(SERVER_COUNTERS)))
    return dict(zip(SERVER_COUNTERS, list(c)))


def nls_server_destroy(s) -> None:
    _gcheck(load_library().nls_server_destroy(s))


# ------------------------------------------------------------- torch helpers

class Solver:
    """A handle bound to a torch CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None, mem_cap_bytes: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the batched solver has no CPU path")
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.h = nls_batch_create(device, self.stream.cuda_stream, mem_cap_bytes)

    def close(self) -> None:
        if self.h:
            nls_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option: int, value: int) -> None:
        nls_set_option(self.h, option, value)

    def launches(self) -> int:
        return nls_launch_count(self.h)

    def submit(self, family: int, params, u, alg: int, abstol: float = 1e-10, maxiters: int = 50,
               outputs=None) -> int:
        """Enqueue; ``u`` ([n, B] float64 CUDA, contiguous) is overwritten with the roots.
        ``outputs`` = (status, iters, resid, nfev[, ngrad]) tensors (or None
        entries), or None."""
        n, B = u.shape
        ptrs = [0, 0, 0, 0, 0]
        if outputs is not None:
            for i, t in enumerate(outputs):
                ptrs[i] = t.data_ptr() if t is not None else 0
        p = params.data_ptr() if params is not None and params.numel() else 0
        return nls_solve(self.h, family, p, u.data_ptr(), n, B, alg, abstol, maxiters, *ptrs)

    def flush(self) -> None:
        nls_flush(self.h)

    def autotune(self, family: int, params, u, alg: int, abstol: float = 1e-10,
                 maxiters: int = 50) -> int:
        n, B = u.shape
        p = params.data_ptr() if params is not None and params.numel() else 0
        return nls_autotune(self.h, family, p, u.data_ptr(), n, B, alg, abstol, maxiters)

    def wait(self, req: int, timeout_ms: int = -1):
        return nls_status(self.h, req, timeout_ms)


def solve(family: int, params, u0, alg: int = NLS_NEWTON, abstol: float = 1e-10,
          maxiters: int = 50, solver: Solver | None = None):
    """Solve a batch held in torch CUDA tensors (params [E, B], u0 [n, B], float64).

    Returns (u, status, iters, resid_inf, nfev, solved)."""
    import torch
    s = solver or Solver(u0.device.index or 0)
    u = u0.detach().clone().contiguous()
    n, B = u.shape
    dev = u.device
    status = torch.empty(B, dtype=torch.int32, device=dev)
    iters = torch.empty(B, dtype=torch.int32, device=dev)
    resid = torch.empty(B, dtype=torch.float64, device=dev)
    nfev = torch.empty(B, dtype=torch.int32, device=dev)
    p = params.contiguous() if params is not None else None
    req = s.submit(family, p, u, alg, abstol, maxiters, (status, iters, resid, nfev))
    solved = s.wait(req)
    return u, status, iters, resid, nfev, solved
