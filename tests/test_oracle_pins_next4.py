"""Pins of the oracle's higher-order, multi-step and quasi-Newton solvers
(Halley, Eq. 3; Potra-Ptak, Eq. 4; Broyden and modified Broyden, Tab. 1) to
facts other than the oracle itself (no GPU needed):

- exact rational iterates of the classic scalar forms of each method,
  computed with Python fractions (Halley's x - 2 f f' / (2 f'^2 - f f''),
  the two-substep Potra-Ptak map, the secant method);
- the second directional derivative against central second differences
  (exact, up to rounding, for residuals that are cubic polynomials along t);
- the Broyden update's defining properties: the secant condition, no change
  on the orthogonal complement of the step, and the least-change norm;
- Gay's theorem: Broyden's good method ends on a linear system within 2n
  steps;
- the pinned roots (closed forms, Cardano, bisection, the Rosenbrock ones).
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O
from paper_2403_16341_gb300 import inputs as I

CUBIC, BRATU, SQUARE, ROSEN = 0, 1, 2, 3
NEW_ALGS = (O.ALG_POTRA_PTAK, O.ALG_HALLEY, O.ALG_BROYDEN, O.ALG_MOD_BROYDEN)


def iterates(family, p, u0, alg, k):
    """u after exactly k loop passes (abstol 0 keeps the loop going)."""
    u, st, it, _, _ = O.solve_one(family, p, u0, alg, abstol=0.0, maxiters=k)
    assert it == k, (st, it)
    return u


def close(x, exact, ulps=8):
    exact = float(exact)
    return abs(x - exact) <= ulps * np.spacing(abs(exact)) + 1e-300


# ---------------------------------------------------------------- H a a

@pytest.mark.parametrize("family,n", [(CUBIC, 5), (SQUARE, 4), (ROSEN, 6), (BRATU, 5)])
def test_hvv_matches_central_second_difference(family, n):
    rng = np.random.default_rng(3 + family)
    E = {CUBIC: n * n + n, BRATU: 1, SQUARE: n, ROSEN: 0}[family]
    p = rng.uniform(0.5, 2.0, max(E, 1))
    u = rng.uniform(-1.0, 1.0, n)
    a = rng.uniform(-1.0, 1.0, n)
    h = O.hvv(family, p, u, a)
    # along t the cubic, square and Rosenbrock residuals are polynomials of
    # degree <= 3, so the central second difference is exact up to rounding
    t = 1e-2 if family != BRATU else 1e-4
    fd = (O.residual(family, p, u + t * a) - 2 * O.residual(family, p, u)
          + O.residual(family, p, u - t * a)) / (t * t)
    tol = 1e-9 if family != BRATU else 1e-5
    np.testing.assert_allclose(h, fd, rtol=tol, atol=tol * np.abs(fd).max())
    # quadratic in a: H (2a)(2a) = 4 H a a
    np.testing.assert_allclose(O.hvv(family, p, u, 2 * a), 4 * h, rtol=1e-15, atol=0)


# ---------------------------------------------------------------- Halley (Eq. 3)

def halley_scalar(f, df, d2f, x):
    fx, d1, d2 = f(x), df(x), d2f(x)
    return x - 2 * fx * d1 / (2 * d1 * d1 - fx * d2)


def test_halley_square_is_the_rational_sqrt_map():
    # f = x^2 - p: Halley's iterate is x (x^2 + 3p) / (3x^2 + p)
    p = [Fr(2), Fr(3), Fr(7, 4), Fr(10)]
    x = [Fr(1), Fr(5, 2), Fr(1, 2), Fr(4)]
    for k in range(1, 4):
        x = [xi * (xi * xi + 3 * pi) / (3 * xi * xi + pi) for xi, pi in zip(x, p)]
        u = iterates(SQUARE, [float(v) for v in p], [1.0, 2.5, 0.5, 4.0], O.ALG_HALLEY, k)
        assert all(close(ui, xi) for ui, xi in zip(u, x)), (k, u, [float(v) for v in x])


def test_halley_diagonal_cubic_is_scalar_halley():
    # A diagonal decouples the cubic family into n scalar equations
    # f_i(x) = a_i x + x^3 - b_i; each component follows x - 2 f f' / (2 f'^2 - f f'')
    n = 3
    a = [Fr(3), Fr(5, 2), Fr(4)]
    b = [Fr(5), Fr(-3), Fr(1, 2)]
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] = float(a[i])
    p = np.concatenate([A.ravel(), [float(v) for v in b]])
    x = [Fr(0)] * n
    for k in range(1, 4):
        x = [halley_scalar(lambda t, i=i: a[i] * t + t ** 3 - b[i],
                           lambda t, i=i: a[i] + 3 * t * t,
                           lambda t: 6 * t, x[i]) for i in range(n)]
        u = iterates(CUBIC, p, np.zeros(n), O.ALG_HALLEY, k)
        assert all(close(ui, xi, 16) for ui, xi in zip(u, x)), (k, u, [float(v) for v in x])


def test_halley_zero_denominator_takes_the_newton_component():
    # component 0 starts at its root: a_0 = 0 and b_0 = 0, so the elementwise
    # quotient is 0/0; the step component is a_0 = 0 and u_0 stays exactly 2
    u, st, it, r, _ = O.solve_one(SQUARE, [4.0, 2.0], [2.0, 1.0], O.ALG_HALLEY, abstol=1e-14)
    assert st == O.ST_SUCCESS and u[0] == 2.0
    assert abs(u[1] - math.sqrt(2.0)) < 1e-15


def test_halley_converges_cubically_on_cubic():
    # e_{k+1} / e_k^3 stays bounded (Newton's e_{k+1} / e_k^2 would not drop as fast)
    n = 1
    p = [2.0, 3.0]  # f = 2x + x^3 - 3, root 1
    errs = []
    for k in range(1, 4):
        u = iterates(CUBIC, p, [3.0], O.ALG_HALLEY, k)
        errs.append(abs(u[0] - 1.0))
    assert errs[1] < errs[0] ** 3 * 5 and errs[2] <= max(errs[1] ** 3 * 5, 2.3e-16)


# ---------------------------------------------------------------- Potra-Ptak (Eq. 4)

def test_potra_ptak_square_rational_map():
    # y = x - f(x)/f'(x), x' = y - f(y)/f'(x), f = x^2 - p, f' = 2x
    p = [Fr(2), Fr(9), Fr(1, 3)]
    x = [Fr(1), Fr(5), Fr(2)]
    for k in range(1, 4):
        nx = []
        for xi, pi in zip(x, p):
            y = xi - (xi * xi - pi) / (2 * xi)
            nx.append(y - (y * y - pi) / (2 * xi))
        x = nx
        u = iterates(SQUARE, [float(v) for v in p], [1.0, 5.0, 2.0], O.ALG_POTRA_PTAK, k)
        assert all(close(ui, xi, 16) for ui, xi in zip(u, x)), (k, u, [float(v) for v in x])


def test_potra_ptak_diagonal_cubic_uses_the_same_jacobian_twice():
    n = 2
    a = [Fr(3), Fr(7, 2)]
    b = [Fr(4), Fr(-1)]
    p = np.concatenate([np.diag([float(v) for v in a]).ravel(), [float(v) for v in b]])
    x = [Fr(0), Fr(0)]
    for k in range(1, 4):
        nx = []
        for i in range(n):
            f = lambda t: a[i] * t + t ** 3 - b[i]  # noqa: E731
            d = a[i] + 3 * x[i] * x[i]
            y = x[i] - f(x[i]) / d
            nx.append(y - f(y) / d)
        x = nx
        u = iterates(CUBIC, p, np.zeros(n), O.ALG_POTRA_PTAK, k)
        assert all(close(ui, xi, 16) for ui, xi in zip(u, x)), (k, u, [float(v) for v in x])


def test_potra_ptak_counts_two_residuals_per_pass():
    _, st, it, _, nfev = O.solve_one(SQUARE, [2.0, 5.0], [1.0, 2.0], O.ALG_POTRA_PTAK,
                                     abstol=1e-13)
    assert st == O.ST_SUCCESS and nfev == 1 + 2 * it


# ---------------------------------------------------------------- Broyden (Tab. 1)

def test_broyden_update_secant_least_change():
    rng = np.random.default_rng(11)
    for n in (1, 3, 8):
        B = rng.standard_normal((n, n))
        du = rng.standard_normal(n)
        df = rng.standard_normal(n)
        B1 = O.broyden_update(B, du, df)
        # secant condition
        np.testing.assert_allclose(B1 @ du, df, rtol=1e-12, atol=1e-12)
        # no change on vectors orthogonal to du
        for _ in range(3):
            v = rng.standard_normal(n)
            v -= (v @ du) / (du @ du) * du
            np.testing.assert_allclose(B1 @ v, B @ v, rtol=1e-12, atol=1e-12)
        # rank one with the least Frobenius norm among secant updates
        D = B1 - B
        s = np.linalg.svd(D, compute_uv=False)
        assert s[1:].max(initial=0.0) <= 1e-12 * s[0]
        np.testing.assert_allclose(np.linalg.norm(D), np.linalg.norm(df - B @ du)
                                   / np.linalg.norm(du), rtol=1e-12)
    # a zero step leaves B as it is
    B = rng.standard_normal((3, 3))
    np.testing.assert_array_equal(O.broyden_update(B, np.zeros(3), np.ones(3)), B)


def test_broyden_gay_finite_termination_on_linear_systems():
    # Gay (1979): good Broyden with any nonsingular start ends on A x = c in at
    # most 2n steps.  The steps are composed from the oracle's update and LU.
    rng = np.random.default_rng(5)
    for n in (2, 4, 6):
        A = rng.standard_normal((n, n)) + n * np.eye(n)
        c = rng.standard_normal(n)
        x = np.zeros(n)
        B = np.eye(n)
        F = A @ x - c
        for _ in range(2 * n):
            LU, piv, info = O.lu_factor(B)
            assert info == 0
            d = O.lu_solve(LU, piv, -F)
            x = x + d
            F1 = A @ x - c
            B = O.broyden_update(B, d, F1 - F)
            F = F1
        assert np.abs(F).max() <= 1e-9 * (np.abs(c).max() + 1), np.abs(F).max()


def secant_iterates(f, x0, x1, k):
    xs = [x0, x1]
    while len(xs) < k + 1:
        a, b = xs[-2], xs[-1]
        xs.append(b - f(b) * (b - a) / (f(b) - f(a)))
    return xs


@pytest.mark.parametrize("alg", [O.ALG_BROYDEN, O.ALG_MOD_BROYDEN])
def test_broyden_scalar_is_the_secant_method(alg):
    # n = 1: B_{k+1} = (f_{k+1} - f_k) / (x_{k+1} - x_k), so after the first
    # step (identity: x1 = x0 - f0; true Jacobian: the Newton step) every step
    # is a secant step
    p = Fr(3)
    f = lambda t: t * t - p  # noqa: E731
    x0 = Fr(2)
    x1 = x0 - f(x0) if alg == O.ALG_BROYDEN else x0 - f(x0) / (2 * x0)
    xs = secant_iterates(f, x0, x1, 5)
    for k in range(1, 6):
        u = iterates(SQUARE, [3.0], [2.0], alg, k)
        assert close(u[0], xs[k], 16), (k, u[0], float(xs[k]))


def test_mod_broyden_first_step_is_newton():
    b = I.cubic_batch(4, 8, seed=21)
    for k in range(8):
        p = b.params[:, k]
        u0 = b.u0[:, k]
        uN = iterates(CUBIC, p, u0, O.ALG_NEWTON, 1)
        uB = iterates(CUBIC, p, u0, O.ALG_MOD_BROYDEN, 1)
        np.testing.assert_array_equal(uN, uB)


# ---------------------------------------------------------------- roots

def cardano(a, b):
    # the real root of x^3 + a x - b = 0 for a > 0
    q = math.sqrt(b * b / 4 + a ** 3 / 27)
    return math.copysign(abs(b / 2 + q) ** (1 / 3), b / 2 + q) + \
        math.copysign(abs(b / 2 - q) ** (1 / 3), b / 2 - q)


@pytest.mark.parametrize("alg", [O.ALG_POTRA_PTAK, O.ALG_HALLEY, O.ALG_MOD_BROYDEN])
def test_diagonal_cubic_reaches_cardano_root(alg):
    rng = np.random.default_rng(2)
    n = 6
    a = rng.uniform(2.0, 4.0, n)
    b = rng.uniform(-5.0, 5.0, n)
    p = np.concatenate([np.diag(a).ravel(), b])
    exact = np.array([cardano(ai, bi) for ai, bi in zip(a, b)])
    # a start near the root: these are local methods (from u0 = 0 the frozen
    # Jacobian of Potra-Ptak's second substep overshoots and the pass cycles)
    u0 = exact + rng.uniform(-0.3, 0.3, n)
    u, st, it, r, _ = O.solve_one(CUBIC, p, u0, alg, abstol=1e-12, maxiters=100)
    assert st == O.ST_SUCCESS
    np.testing.assert_allclose(u, exact, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("alg", NEW_ALGS)
def test_square_reaches_sqrt(alg):
    b = I.square_batch(4, 64, seed=4)
    u, st, it, r, _ = O.solve_batch(b.family, b.params, b.u0, alg, abstol=1e-12, maxiters=200)
    ok = st == O.ST_SUCCESS
    assert ok.mean() > 0.9
    # u_i^2 = p_i has the two roots +-sqrt(p_i); an overshooting step may land on either
    np.testing.assert_allclose(np.abs(u[:, ok]), np.sqrt(b.params[:, ok]), rtol=0, atol=1.01e-12)


@pytest.mark.parametrize("alg", [O.ALG_POTRA_PTAK, O.ALG_HALLEY])
def test_rosenbrock_paper_starts_reach_ones(alg):
    # Sec. 3.3 starts U[0, 1)^10; the root is the all-ones vector
    b = I.rosenbrock_batch(10, 64, seed=0)
    u, st, it, r, _ = O.solve_batch(b.family, b.params, b.u0, alg, abstol=1e-10, maxiters=200)
    ok = st == O.ST_SUCCESS
    assert ok.mean() > 0.8
    np.testing.assert_allclose(u[:, ok], 1.0, rtol=0, atol=1e-10)


@pytest.mark.parametrize("alg", NEW_ALGS)
def test_bratu_n2_matches_bisection(alg):
    # n = 2, symmetric solution u1 = u2 = v: -9 v + lambda e^v = 0 (lower branch)
    lam = 1.0
    lo, hi = 0.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if -9 * mid + lam * math.exp(mid) > 0:
            lo = mid
        else:
            hi = mid
    u, st, it, r, _ = O.solve_one(BRATU, [lam], [0.0, 0.0], alg, abstol=1e-13, maxiters=100)
    assert st == O.ST_SUCCESS
    np.testing.assert_allclose(u, [lo, lo], rtol=0, atol=1e-14)


# ---------------------------------------------------------------- statuses

def test_singular_statuses():
    # J = diag(2u) = 0 at u0 = 0: the Jacobian methods stop at pass 1
    for alg in (O.ALG_POTRA_PTAK, O.ALG_HALLEY, O.ALG_MOD_BROYDEN):
        _, st, it, _, _ = O.solve_one(SQUARE, [2.0, 3.0], [0.0, 0.0], alg)
        assert st == O.ST_SINGULAR and it == 1
    # u^2 = 3 from u0 = 3 with B_0 = 1: du = -6 lands on -3 where F = 6 again,
    # the secant slope df/du is 0, B_1 = 0 exactly and pass 2 finds it singular
    _, st, it, _, _ = O.solve_one(SQUARE, [3.0], [3.0], O.ALG_BROYDEN)
    assert st == O.ST_SINGULAR and it == 2
