"""Seeded synthetic inputs for batched nonlinear solves F(u; p_k) = 0.

This module is shared by the CUDA path, the tests, the oracle harness and the
benchmark.  It draws random numbers and lays them out; it holds none of the
solver's arithmetic (no residual, Jacobian, factorisation or step).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style so any
instance's draws can be produced independently of the others:

    mix(z)     = SplitMix64 output function of a 64-bit word
    base       = mix(seed * GAMMA + config_id + 1)
    key_k      = mix(base + (k + 1) * GAMMA)         # instance k's stream key
    draw_k[j]  = mix(key_k + (j + 1) * GAMMA)        # j-th 64-bit draw

Uniforms on [0, 1) take the top 53 bits; normals use the Box-Muller pair
(sqrt(-2 ln(1 - u1)) cos(2 pi u2), ... sin(2 pi u2)).

Parameter layout ("SoA", element-major, instance fastest): for a batch of B
instances the parameters are a float64 array ``params[E, B]`` with
``params[e, k]`` the e-th parameter of instance k, and ``u0[n, B]``.

  cubic  (F = A u + u*u*u - b):   e < n*n -> A[i, j] at e = i*n + j (row-major),
                                   e = n*n + i -> b[i];  E = n*n + n
  bratu  (1-D Bratu, Dirichlet 0): e = 0 -> lambda;      E = 1
  square (F = u*u - p):           e = i -> p[i];        E = n
  rosenbrock (Eq. 5):             no parameters;        E = 0

The workloads (``workload_*``) reproduce the synthetic families used to
measure the batched solver: the dense cubic with A = 3 I + G, G ~ N(0, 0.3^2),
the 1-D Bratu problem with lambda ~ U[0.5, 3], the generalized Rosenbrock
problem of Sec. 3.3 and an uneven mix of sizes 2..32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

FAMILY_CUBIC = 0
FAMILY_BRATU = 1
FAMILY_SQUARE = 2
FAMILY_ROSENBROCK = 3
FAMILY_NAMES = {FAMILY_CUBIC: "cubic", FAMILY_BRATU: "bratu",
                FAMILY_SQUARE: "square", FAMILY_ROSENBROCK: "rosenbrock"}


def n_params(family: int, n: int) -> int:
    """Number of float64 parameters E per instance for a family of size n."""
    if family == FAMILY_CUBIC:
        return n * n + n
    if family == FAMILY_BRATU:
        return 1
    if family == FAMILY_SQUARE:
        return n
    if family == FAMILY_ROSENBROCK:
        return 0
    raise ValueError(f"unknown family {family}")


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_keys(seed: int, config_id: int, instances: np.ndarray) -> np.ndarray:
    """Per-instance stream keys key_k for the given instance indices."""
    with np.errstate(over="ignore"):
        base = _mix(np.uint64(seed) * GAMMA + np.uint64(config_id + 1))
        k = np.asarray(instances, dtype=np.uint64)
        return _mix(base + (k + np.uint64(1)) * GAMMA)


def raw_draws(keys: np.ndarray, j0: int, m: int) -> np.ndarray:
    """Draws j0 .. j0+m-1 of each stream: uint64 array [len(keys), m]."""
    j = np.arange(j0 + 1, j0 + m + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(keys[:, None] + j[None, :] * GAMMA)


def uniforms(keys: np.ndarray, j0: int, m: int) -> np.ndarray:
    """m uniforms on [0, 1) per stream, from draws j0 ..; float64 [K, m]."""
    return (raw_draws(keys, j0, m) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(keys: np.ndarray, j0: int, m: int) -> np.ndarray:
    """m standard normals per stream (Box-Muller), consuming 2*ceil(m/2) draws."""
    pairs = (m + 1) // 2
    u = uniforms(keys, j0, 2 * pairs)
    r = np.sqrt(-2.0 * np.log1p(-u[:, 0::2]))
    t = 2.0 * math.pi * u[:, 1::2]
    z = np.empty((keys.shape[0], 2 * pairs))
    z[:, 0::2] = r * np.cos(t)
    z[:, 1::2] = r * np.sin(t)
    return z[:, :m]


def _draws_for_normals(m: int) -> int:
    return 2 * ((m + 1) // 2)


# --------------------------------------------------------------------------
# Per-family draws (instance-level, layout-free)
# --------------------------------------------------------------------------

def cubic_instances(keys: np.ndarray, n: int, b_half_width: float,
                    g_sigma: float = 0.3, max_redraws: int = 64):
    """A = 3 I + G (G ~ N(0, g_sigma^2)), b ~ U[-w, w]^n for each stream key.

    The draw order per instance is: attempt 0's n*n normals, then n uniforms
    for b, then (only if sym(A) is not positive definite) further attempts of
    n*n normals each.  sym(A) = (A + A^T)/2 positive definite makes
    F = A u + u^3 - b strictly monotone, so its root is unique; it is checked
    with a Cholesky factorisation and A is redrawn from the same stream until
    it holds.  Returns (A [K, n, n], b [K, n], redraws [K]).
    """
    K = keys.shape[0]
    dn = _draws_for_normals(n * n)
    G = normals(keys, 0, n * n).reshape(K, n, n) * g_sigma
    b = (2.0 * uniforms(keys, dn, n) - 1.0) * b_half_width
    A = G + 3.0 * np.eye(n)[None]
    redraws = np.zeros(K, dtype=np.int32)
    j_next = dn + n
    for _ in range(max_redraws):
        bad = ~_is_spd(0.5 * (A + np.transpose(A, (0, 2, 1))))
        if not bad.any():
            break
        idx = np.nonzero(bad)[0]
        G2 = normals(keys[idx], j_next, n * n).reshape(idx.size, n, n) * g_sigma
        A[idx] = G2 + 3.0 * np.eye(n)[None]
        redraws[idx] += 1
        j_next += dn
    else:
        raise RuntimeError("could not draw a monotone cubic instance")
    return A, b, redraws


def _is_spd(S: np.ndarray) -> np.ndarray:
    ok = np.ones(S.shape[0], dtype=bool)
    chunk = 1 << 16
    for s in range(0, S.shape[0], chunk):
        ok[s:s + chunk] = np.linalg.eigvalsh(S[s:s + chunk])[:, 0] > 0.0
    return ok


def bratu_lambdas(keys: np.ndarray, lo: float = 0.5, hi: float = 3.0) -> np.ndarray:
    return lo + (hi - lo) * uniforms(keys, 0, 1)[:, 0]


# --------------------------------------------------------------------------
# Batches in the SoA layout
# --------------------------------------------------------------------------

@dataclass
class Batch:
    """One uniform-size batch: family, n, params[E, B], u0[n, B] (float64)."""
    family: int
    n: int
    params: np.ndarray
    u0: np.ndarray
    instance_ids: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def batch(self) -> int:
        return self.u0.shape[1]


def cubic_g_sigma(n: int) -> float:
    """Standard deviation of G: 0.3 up to n = 32 (all benchmark sizes); above
    that 0.3 sqrt(32 / n), which keeps the spectral edge of sym(G) (about
    0.42 sqrt(n) sigma / 0.3) below 3 so that sym(A) stays positive definite."""
    return 0.3 if n <= 32 else 0.3 * math.sqrt(32.0 / n)


def cubic_batch(n: int, B: int, seed: int = 0, config_id: int = 0,
                b_half_width: float = 2.0, instances: np.ndarray | None = None) -> Batch:
    ids = np.arange(B, dtype=np.int64) if instances is None else np.asarray(instances)
    keys = stream_keys(seed, config_id, ids)
    A, b, redraws = cubic_instances(keys, n, b_half_width, g_sigma=cubic_g_sigma(n))
    K = ids.size
    params = np.empty((n * n + n, K))
    params[: n * n] = A.reshape(K, n * n).T
    params[n * n:] = b.T
    return Batch(FAMILY_CUBIC, n, np.ascontiguousarray(params), np.zeros((n, K)), ids,
                 {"redraws": int(redraws.sum())})


def bratu_batch(n: int, B: int, seed: int = 0, config_id: int = 0,
                instances: np.ndarray | None = None) -> Batch:
    ids = np.arange(B, dtype=np.int64) if instances is None else np.asarray(instances)
    keys = stream_keys(seed, config_id, ids)
    lam = bratu_lambdas(keys)
    return Batch(FAMILY_BRATU, n, lam[None, :].copy(), np.zeros((n, ids.size)), ids)


def square_batch(n: int, B: int, seed: int = 0, config_id: int = 90,
                 lo: float = 0.25, hi: float = 9.0, u0_value: float = 1.0) -> Batch:
    keys = stream_keys(seed, config_id, np.arange(B))
    p = lo + (hi - lo) * uniforms(keys, 0, n)
    return Batch(FAMILY_SQUARE, n, np.ascontiguousarray(p.T), np.full((n, B), u0_value))


def rosenbrock_batch(n: int, B: int, seed: int = 0, config_id: int = 91) -> Batch:
    """u0 ~ U[0, 1]^n per instance, as in the Sec. 3.3 GPU example."""
    keys = stream_keys(seed, config_id, np.arange(B))
    u0 = uniforms(keys, 0, n)
    return Batch(FAMILY_ROSENBROCK, n, np.zeros((0, B)), np.ascontiguousarray(u0.T))


def lognormal_sizes(keys: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """n = floor(exp(U[ln lo, ln(hi + 1)))) in {lo..hi} (log-uniform sizes)."""
    u = uniforms(keys, 0, 1)[:, 0]
    n = np.floor(np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))).astype(np.int64)
    return np.clip(n, lo, hi)


def uneven_batches(B: int, seed: int = 0, config_id: int = 2, n_lo: int = 2, n_hi: int = 32,
                   b_half_width: float = 2.0) -> list[Batch]:
    """Uneven mix: instance k has n_k log-uniform in {n_lo..n_hi} and family
    k mod 2 (0 cubic, 1 Bratu); instances are grouped into one Batch per
    (family, n), each remembering its original instance ids."""
    ids = np.arange(B, dtype=np.int64)
    size_keys = stream_keys(seed, config_id + 1000, ids)
    sizes = lognormal_sizes(size_keys, n_lo, n_hi)
    fam = (ids % 2).astype(np.int64)
    out = []
    for f in (FAMILY_CUBIC, FAMILY_BRATU):
        for n in range(n_lo, n_hi + 1):
            sel = ids[(fam == f) & (sizes == n)]
            if sel.size == 0:
                continue
            if f == FAMILY_CUBIC:
                out.append(cubic_batch(n, sel.size, seed, config_id, b_half_width, instances=sel))
            else:
                out.append(bratu_batch(n, sel.size, seed, config_id, instances=sel))
    return out


def bratu_uniform_n_batches(B: int, n_lo: int, n_hi: int, seed: int = 0,
                            config_id: int = 4) -> list[Batch]:
    """B Bratu instances with n uniform on {n_lo..n_hi}, grouped by n."""
    ids = np.arange(B, dtype=np.int64)
    u = uniforms(stream_keys(seed, config_id + 1000, ids), 0, 1)[:, 0]
    sizes = n_lo + np.minimum((u * (n_hi - n_lo + 1)).astype(np.int64), n_hi - n_lo)
    out = []
    for n in range(n_lo, n_hi + 1):
        sel = ids[sizes == n]
        if sel.size:
            out.append(bratu_batch(n, sel.size, seed, config_id, instances=sel))
    return out


# Named workloads ------------------------------------------------------------

def workload_cubic_n3(seed: int = 0) -> Batch:
    """1,024 cubic instances, n = 3, b ~ U[-2, 2]^3, u0 = 0."""
    return cubic_batch(3, 1024, seed, config_id=0, b_half_width=2.0)


def workload_cubic_n8(B: int = 1 << 20, seed: int = 0) -> Batch:
    """Cubic instances with n = 8, b ~ U[-5, 5]^8, u0 = 0 (2^20 by default)."""
    return cubic_batch(8, B, seed, config_id=1, b_half_width=5.0)


def workload_uneven(B: int = 1 << 18, seed: int = 0) -> list[Batch]:
    """2^18 instances, n log-uniform in 2..32, half cubic and half Bratu."""
    return uneven_batches(B, seed, config_id=2)


def workload_bratu_large(B: int = 16384, seed: int = 0) -> list[Batch]:
    """16,384 Bratu instances with n uniform in 64..128."""
    return bratu_uniform_n_batches(B, 64, 128, seed, config_id=4)


# Serving workload -----------------------------------------------------------

@dataclass
class ServingRequest:
    family: int
    n: int
    batch: int
    params: np.ndarray  # [E, batch], float64, C-contiguous
    arrival: float      # seconds after the start of the stream


def serving_payloads(count: int, seed: int = 0, config_id: int = 3,
                     max_batch: int = 4096) -> list[Batch]:
    """`count` distinct request payloads: batch size floor(exp(U[0, ln(max_batch + 1))))
    in 1..max_batch (log-uniform), n uniform in {3, 8, 16, 32}, family uniform
    in {cubic (A = 3 I + G, b ~ U[-2, 2]^n), Bratu (lambda ~ U[0.5, 3])}, u0 = 0."""
    keys = stream_keys(seed, config_id + 2000, np.arange(count))
    u = uniforms(keys, 0, 3)
    sizes = np.minimum(np.floor(np.exp(u[:, 0] * math.log(max_batch + 1))).astype(np.int64),
                       max_batch)
    sizes = np.maximum(sizes, 1)
    ns = np.array([3, 8, 16, 32])[np.minimum((u[:, 1] * 4).astype(np.int64), 3)]
    fams = (u[:, 2] < 0.5).astype(np.int64)  # 0 cubic, 1 Bratu
    out, start = [], 0
    for r in range(count):
        ids = np.arange(start, start + sizes[r])
        start += sizes[r]
        if fams[r] == FAMILY_CUBIC:
            out.append(cubic_batch(int(ns[r]), int(sizes[r]), seed, config_id, 2.0, instances=ids))
        else:
            out.append(bratu_batch(int(ns[r]), int(sizes[r]), seed, config_id, instances=ids))
    return out


def poisson_arrivals(count: int, rate: float, seed: int = 0, config_id: int = 3) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with `rate` requests/s."""
    keys = stream_keys(seed, config_id + 3000, np.arange(count))
    gaps = -np.log1p(-uniforms(keys, 0, 1)[:, 0]) / rate
    return np.cumsum(gaps)
