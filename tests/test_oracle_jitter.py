"""The oracle's test-only step perturbation ("jitter") and the batch wrapper's
handling of u0, checked without a GPU.

The GPU parity tests use jittered oracle runs to tell instances whose outcome
is decided by rounding from those the method decides, so the jitter must do
exactly what it says: multiply each component of each computed step by
1 + eps or 1 - eps, reproducibly per (seed, instance), and nothing at all
when eps = 0."""
import ctypes

import numpy as np
import pytest

import oracle as O
import oracle.oracle as OO
from paper_2403_16341_gb300 import inputs as I


def _raw_jitter(b, alg, eps, seed, maxiters=50):
    # the jittered C entry called directly (solve_batch takes the plain
    # entry when jitter == 0)
    lib = OO._load()
    n, B = b.u0.shape
    P = np.ascontiguousarray(b.params.T) if b.params.size else np.zeros((1, 1))
    U = np.array(b.u0.T, order="C", copy=True)
    st, it, nf = (np.zeros(B, np.int32) for _ in range(3))
    rs = np.zeros(B)
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    lib.oracle_solve_range_jitter(b.family, n, 0, B, dp(P), dp(U), alg, 1e-10, maxiters, ip(st),
                                  ip(it), dp(rs), ip(nf), eps, seed)
    return U.T, st, it


@pytest.mark.parametrize("alg", [O.ALG_NEWTON, O.ALG_NEWTON_BACKTRACK, O.ALG_TRUST_DOGLEG,
                                 O.ALG_POTRA_PTAK, O.ALG_HALLEY, O.ALG_BROYDEN,
                                 O.ALG_MOD_BROYDEN])
def test_zero_jitter_is_the_plain_solver(alg):
    b = I.cubic_batch(5, 64, config_id=2)
    u, st, it, _, _ = O.solve_batch(b.family, b.params, b.u0, alg)
    uj, stj, itj = _raw_jitter(b, alg, 0.0, 12345)
    np.testing.assert_array_equal(uj, u)
    np.testing.assert_array_equal(stj, st)
    np.testing.assert_array_equal(itj, it)


def test_jitter_scales_each_step_component():
    # one Newton pass on u.*u = p from u0 = 1: the exact step is (p - 1) / 2,
    # and the jittered pass must land on u0 + step (1 +- eps), componentwise
    b = I.square_batch(6, 200)
    eps = 1e-3
    u1, *_ = O.solve_batch(b.family, b.params, b.u0, O.ALG_NEWTON, 1e-10, 1, jitter=eps, seed=7)
    step = (b.params - 1.0) / 2.0
    ratio = (u1 - b.u0) / step
    dev = np.abs(np.abs(ratio - 1.0) - eps)
    assert dev.max() < 1e-12
    signs = np.sign(ratio - 1.0)
    assert 0.4 < (signs > 0).mean() < 0.6  # both signs, about equally often
    # reproducible per (seed, instance), whatever the split over threads
    u2, *_ = O.solve_batch(b.family, b.params, b.u0, O.ALG_NEWTON, 1e-10, 1, jitter=eps, seed=7,
                           threads=4)
    np.testing.assert_array_equal(u2, u1)
    half = I.Batch(b.family, b.n, b.params[:, :100].copy(), b.u0[:, :100].copy())
    u3, *_ = O.solve_batch(half.family, half.params, half.u0, O.ALG_NEWTON, 1e-10, 1,
                           jitter=eps, seed=7)
    np.testing.assert_array_equal(u3, u1[:, :100])
    # another seed, other signs
    u4, *_ = O.solve_batch(b.family, b.params, b.u0, O.ALG_NEWTON, 1e-10, 1, jitter=eps, seed=8)
    assert (np.sign((u4 - b.u0) / step - 1.0) != signs).mean() > 0.3


def test_jitter_does_not_change_well_posed_outcomes():
    # Newton with backtracking on the cubic family converges robustly: steps
    # perturbed by 1e-6 still reach every root (Newton's self-correction)
    b = I.cubic_batch(8, 300, config_id=1, b_half_width=5.0)
    u, st, *_ = O.solve_batch(b.family, b.params, b.u0, O.ALG_NEWTON_BACKTRACK)
    uj, stj, *_ = O.solve_batch(b.family, b.params, b.u0, O.ALG_NEWTON_BACKTRACK, jitter=1e-6,
                                seed=3)
    assert (st == 0).all() and (stj == 0).all()
    assert np.abs(uj - u).max() < 1e-9


@pytest.mark.parametrize("n", [1, 3])
def test_solve_batch_leaves_u0_alone(n):
    # for n = 1 the transposed u0 is already contiguous: the wrapper must
    # still solve in a copy and not write the roots into the caller's u0
    b = I.square_batch(n, 16)
    before = b.u0.copy()
    u, st, *_ = O.solve_batch(b.family, b.params, b.u0, O.ALG_NEWTON)
    np.testing.assert_array_equal(b.u0, before)
    assert (st == 0).all() and not np.array_equal(u, before)
