"""ctypes binding of the C oracle (``nls_oracle.c``).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the bench).

Batches are passed in the element-major layout the GPU library uses
(``params[E, B]``, ``u0[n, B]``); this wrapper transposes them to the
instance-major layout the C code walks.  ``solve_batch`` can split a batch
over host threads (ctypes releases the GIL during the C call).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ALG_NEWTON, ALG_NEWTON_BACKTRACK, ALG_TRUST_DOGLEG = 0, 1, 2
ALG_POTRA_PTAK, ALG_HALLEY, ALG_BROYDEN, ALG_MOD_BROYDEN = 4, 5, 6, 7
ALG_TRUST_DOGLEG_NW = 8  # trust region with the NocedalWright radius update
ST_SUCCESS, ST_MAXITERS, ST_SINGULAR, ST_NONFINITE, ST_LS_FAILED, ST_TR_STALLED = range(6)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nls_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_residual.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
            lib.oracle_jacobian.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
            lib.oracle_lu_factor.argtypes = [ctypes.c_int, _D, _I]
            lib.oracle_lu_factor.restype = ctypes.c_int
            lib.oracle_lu_solve.argtypes = [ctypes.c_int, _D, _I, _D, _D]
            lib.oracle_dogleg.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double, _D]
            lib.oracle_dogleg.restype = ctypes.c_int
            lib.oracle_solve_trace.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_int, _I, _D, _I, _D, _I,
                                               _I, _D, _D, _D]
            lib.oracle_solve_trace.restype = ctypes.c_int
            lib.oracle_solve_range.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_long,
                                               ctypes.c_long, _D, _D, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_int, _I, _I, _D, _I]
            lib.oracle_solve_range_jitter.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_long, ctypes.c_long, _D, _D, ctypes.c_int,
                ctypes.c_double, ctypes.c_int, _I, _I, _D, _I, ctypes.c_double, ctypes.c_uint64]
            lib.oracle_polish.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int]
            lib.oracle_polish.restype = ctypes.c_double
            lib.oracle_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
            lib.oracle_adjoint.restype = ctypes.c_int
            lib.oracle_hvv.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
            lib.oracle_broyden_update.argtypes = [ctypes.c_int, _D, _D, _D]
            lib.oracle_n_params.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.oracle_n_params.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(_I)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def residual(family: int, p, u) -> np.ndarray:
    p, u = _f64(p), _f64(u)
    F = np.empty_like(u)
    _load().oracle_residual(family, u.size, _dp(p), _dp(u), _dp(F))
    return F


def jacobian(family: int, p, u) -> np.ndarray:
    p, u = _f64(p), _f64(u)
    J = np.empty((u.size, u.size))
    _load().oracle_jacobian(family, u.size, _dp(p), _dp(u), _dp(J))
    return J


def hvv(family: int, p, u, a) -> np.ndarray:
    """d^2/dt^2 F(u + t a) at t = 0 (the H a a term of Halley's method)."""
    p = _f64(p) if np.size(p) else np.zeros(1)
    u, a = _f64(u), _f64(a)
    h = np.empty_like(u)
    _load().oracle_hvv(family, u.size, _dp(p), _dp(u), _dp(a), _dp(h))
    return h


def broyden_update(B, du, df) -> np.ndarray:
    """Good Broyden rank-one update of the Jacobian approximation B."""
    B = _f64(B).copy()
    du, df = _f64(du), _f64(df)
    _load().oracle_broyden_update(du.size, _dp(B), _dp(du), _dp(df))
    return B


def lu_factor(A):
    """Returns (LU, piv, info): info = 0 or 1 + index of the failed pivot."""
    LU = _f64(A).copy()
    n = LU.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    info = _load().oracle_lu_factor(n, _dp(LU), _ip(piv))
    return LU, piv, info


def lu_solve(LU, piv, rhs) -> np.ndarray:
    LU, rhs = _f64(LU), _f64(rhs)
    piv = np.ascontiguousarray(piv, dtype=np.int32)
    x = np.empty_like(rhs)
    _load().oracle_lu_solve(rhs.size, _dp(LU), _ip(piv), _dp(rhs), _dp(x))
    return x


def dogleg(J, F, dN, Delta: float):
    """Returns (step, branch) with branch 0 Newton, 1 boundary along -g, 2 dogleg."""
    J, F, dN = _f64(J), _f64(F), _f64(dN)
    d = np.empty_like(F)
    br = _load().oracle_dogleg(F.size, _dp(J), _dp(F), _dp(dN), float(Delta), _dp(d))
    return d, br


def solve_one(family: int, p, u0, alg: int, abstol: float = 1e-10, maxiters: int = 50):
    """Returns (u, status, iters, resid_inf, nfev) for one instance."""
    r = solve_trace(family, p, u0, alg, abstol, maxiters)
    return r["u"], r["status"], r["iters"], r["resid"], r["nfev"]


def solve_trace(family: int, p, u0, alg: int, abstol: float = 1e-10, maxiters: int = 50) -> dict:
    p = _f64(p) if np.size(p) else np.zeros(1)
    u = _f64(u0).copy()
    m = max(int(maxiters), 1)
    alpha = np.zeros(m)
    rho = np.zeros(m)
    radius = np.zeros(m)
    fnorm = np.zeros(m)
    trials = np.zeros(m, dtype=np.int32)
    branch = np.full(m, -1, dtype=np.int32)
    it, nf = ctypes.c_int(0), ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    st = _load().oracle_solve_trace(family, u.size, _dp(p), _dp(u), alg, float(abstol),
                                    int(maxiters), ctypes.byref(it), ctypes.byref(res),
                                    ctypes.byref(nf), _dp(alpha), _ip(trials), _ip(branch),
                                    _dp(rho), _dp(radius), _dp(fnorm))
    k = it.value
    return {"u": u, "status": st, "iters": k, "resid": res.value, "nfev": nf.value,
            "alpha": alpha[:k], "trials": trials[:k], "branch": branch[:k], "rho": rho[:k],
            "radius": radius[:k], "fnorm": fnorm[:k]}


def solve_batch(family: int, params, u0, alg: int, abstol: float = 1e-10, maxiters: int = 50,
                threads: int = 1, jitter: float = 0.0, seed: int = 0):
    """Solve a batch given element-major params[E, B], u0[n, B].

    jitter > 0 (tests only) multiplies every component of every computed
    step by 1 +- jitter, signs from a stream keyed by (seed, instance).

    Returns (u[n, B], status[B], iters[B], resid[B], nfev[B])."""
    u0 = np.asarray(u0, dtype=np.float64)
    n, B = u0.shape
    params = np.asarray(params, dtype=np.float64).reshape(-1, B)
    P = np.ascontiguousarray(params.T) if params.shape[0] else np.zeros((B, 1))
    U = np.array(u0.T, order="C", copy=True)  # always a copy: the C code writes the roots here
    status = np.zeros(B, dtype=np.int32)
    iters = np.zeros(B, dtype=np.int32)
    nfev = np.zeros(B, dtype=np.int32)
    resid = np.zeros(B)
    lib = _load()
    if lib.oracle_n_params(family, n) == 0:
        P = np.zeros((1, 1))  # no parameters: every instance gets the same unread vector

    def run(k0: int, k1: int) -> None:
        if jitter:
            lib.oracle_solve_range_jitter(family, n, k0, k1, _dp(P), _dp(U), alg, float(abstol),
                                          int(maxiters), _ip(status), _ip(iters), _dp(resid),
                                          _ip(nfev), float(jitter), int(seed))
        else:
            lib.oracle_solve_range(family, n, k0, k1, _dp(P), _dp(U), alg, float(abstol),
                                   int(maxiters), _ip(status), _ip(iters), _dp(resid), _ip(nfev))

    if threads <= 1 or B < 2 * threads:
        run(0, B)
    else:
        bounds = np.linspace(0, B, threads + 1).astype(np.int64)
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda i: run(int(bounds[i]), int(bounds[i + 1])), range(threads)))
    return np.ascontiguousarray(U.T), status, iters, resid, nfev


def polish(family: int, p, u, maxsteps: int = 8):
    """Extra Newton steps while ||F||_inf decreases; returns (u, ||F||_inf)."""
    p = _f64(p) if np.size(p) else np.zeros(1)
    u = _f64(u).copy()
    fn = _load().oracle_polish(family, u.size, _dp(p), _dp(u), int(maxsteps))
    return u, fn


def polish_batch(family: int, params, u, maxsteps: int = 8) -> np.ndarray:
    """Polish every column of u[n, B] (element-major); returns the polished u."""
    u = np.array(u, dtype=np.float64, copy=True)
    n, B = u.shape
    params = np.asarray(params, dtype=np.float64).reshape(-1, B)
    for k in range(B):
        p = params[:, k] if params.shape[0] else np.zeros(1)
        u[:, k], _ = polish(family, p, u[:, k], maxsteps)
    return u


def adjoint(family: int, p, u, w):
    """dL/dtheta at the root u for the cotangent w = dL/du (implicit function
    theorem).  Returns (grad[E], singular)."""
    p = _f64(p) if np.size(p) else np.zeros(1)
    u, w = _f64(u), _f64(w)
    E = _load().oracle_n_params(family, u.size)
    g = np.zeros(max(E, 1))
    rc = _load().oracle_adjoint(family, u.size, _dp(p), _dp(u), _dp(w), _dp(g))
    return g[:E], bool(rc)
