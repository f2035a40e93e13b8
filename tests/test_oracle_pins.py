"""Pins of the FP64 oracle to facts other than itself (no GPU needed).

Each test checks the oracle against something the paper or the mathematics
fixes: closed-form roots, bisection brute force, LAPACK's LU, MINPACK's
hybrid solver (scipy), hand-derived dogleg steps, the Armijo inequality and
the paper's worked examples (fixtures in tests/golden/, each with its
citation).  A dropped term, a wrong sign or index, or a transposed operand
anywhere in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

import oracle as O
from paper_2403_16341_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CUBIC, BRATU, SQUARE, ROSEN = 0, 1, 2, 3
ALGS = (O.ALG_NEWTON, O.ALG_NEWTON_BACKTRACK, O.ALG_TRUST_DOGLEG)


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("alg", ALGS)
def test_square_example_sec2_3(alg):
    g = golden("square_sec2_3.json")
    u, st, it, r, _ = O.solve_one(SQUARE, g["p"], g["u0"], alg, abstol=1e-13)
    assert st == O.ST_SUCCESS
    np.testing.assert_allclose(u, g["root"], rtol=2e-16, atol=0)
    np.testing.assert_allclose(u, np.sqrt(g["p"]), rtol=2e-16)
    # g(u*) = sum u*^2 = sum p, so dg/dp = 1 (the example's gradient)
    assert abs(np.sum(u ** 2) - np.sum(g["p"])) < 1e-13


@pytest.mark.parametrize("alg", ALGS)
def test_square_batch_sqrt(alg):
    b = I.square_batch(5, 300)
    u, st, it, r, _ = O.solve_batch(b.family, b.params, b.u0, alg, abstol=1e-12)
    assert (st == O.ST_SUCCESS).all()
    # |u - sqrt(p)| <= abstol / (2 sqrt(p)) at convergence (p >= 1/4)
    np.testing.assert_allclose(u, np.sqrt(b.params), rtol=0, atol=1.01e-12)


def test_square_from_zero_is_singular():
    # J = diag(2 u) = 0 at u0 = 0
    u, st, it, r, _ = O.solve_one(SQUARE, [2.0, 3.0], [0.0, 0.0], O.ALG_NEWTON)
    assert st == O.ST_SINGULAR and it == 1


def cardano_root(b):
    # the one real root of u^3 + 3u - b = 0
    s = np.sqrt(b * b / 4.0 + 1.0)
    return np.cbrt(b / 2.0 + s) + np.cbrt(b / 2.0 - s)


@pytest.mark.parametrize("alg", ALGS)
def test_cubic_diagonal_cardano(alg):
    n, B = 4, 200
    rng = np.random.default_rng(1)
    bvec = rng.uniform(-5, 5, size=(n, B))
    A = np.tile((3.0 * np.eye(n)).reshape(-1, 1), (1, B))
    params = np.vstack([A, bvec])
    u, st, it, r, _ = O.solve_batch(CUBIC, params, np.zeros((n, B)), alg, abstol=1e-13)
    assert (st == O.ST_SUCCESS).all()
    np.testing.assert_allclose(u, cardano_root(bvec), rtol=1e-13, atol=1e-14)


def bisect_vec(f, lo, hi, iters=200):
    lo, hi = np.array(lo, dtype=float), np.array(hi, dtype=float)
    flo = f(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        left = np.sign(fm) == np.sign(flo)
        lo = np.where(left, mid, lo)
        flo = np.where(left, fm, flo)
        hi = np.where(left, hi, mid)
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("alg", ALGS)
def test_cubic_diagonal_bisection(alg):
    n, B = 6, 100
    rng = np.random.default_rng(2)
    a = rng.uniform(0.2, 5.0, size=(n, B))
    bvec = rng.uniform(-5, 5, size=(n, B))
    A = np.zeros((n * n, B))
    for i in range(n):
        A[i * n + i] = a[i]
    u, st, it, r, _ = O.solve_batch(CUBIC, np.vstack([A, bvec]), np.zeros((n, B)), alg,
                                    abstol=1e-13)
    assert (st == O.ST_SUCCESS).all()
    R = np.maximum(1.0, np.abs(bvec))
    ref = bisect_vec(lambda x: a * x + x ** 3 - bvec, -R, R)
    np.testing.assert_allclose(u, ref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("alg", ALGS)
def test_bratu_n2_bisection(alg):
    # n = 2, h = 1/3: by symmetry u1 = u2 = s with -9 s + lambda e^s = 0
    lam = np.linspace(0.5, 3.0, 11)
    ref = bisect_vec(lambda s: -9.0 * s + lam * np.exp(s), np.zeros_like(lam), np.ones_like(lam))
    params = lam[None, :]
    u, st, it, r, _ = O.solve_batch(BRATU, params, np.zeros((2, lam.size)), alg, abstol=1e-13)
    assert (st == O.ST_SUCCESS).all()
    # |F| <= 1e-13 and |dF/ds| >= 5 on [0, 0.62] bound the error by 2e-14
    np.testing.assert_allclose(u[0], ref, rtol=0, atol=3e-14)
    np.testing.assert_allclose(u[1], ref, rtol=0, atol=3e-14)


def bratu_continuous(x, lam):
    # u(x) = -2 ln( cosh((x - 1/2) t / 2) / cosh(t / 4) ), t = sqrt(2 lam) cosh(t / 4) (lower branch)
    t = scipy.optimize.brentq(lambda t: t - math.sqrt(2 * lam) * math.cosh(t / 4), 0.0, 4.0)
    return -2.0 * np.log(np.cosh((x - 0.5) * t / 2) / np.cosh(t / 4))


@pytest.mark.parametrize("n", [64, 128])
def test_bratu_large_n_matches_continuous_solution(n):
    for lam in (0.5, 1.7, 3.0):
        u, st, it, r, _ = O.solve_one(BRATU, [lam], np.zeros(n), O.ALG_TRUST_DOGLEG)
        assert st == O.ST_SUCCESS
        x = np.arange(1, n + 1) / (n + 1)
        err = np.abs(u - bratu_continuous(x, lam)).max()
        assert err < 2e-4 * (64.0 / n) ** 2 + 1e-6, err


def test_rosenbrock_fig1_example():
    g = golden("rosenbrock_sec2_2_1.json")
    u0 = np.array(g["u0"])
    u, st, it, r, _ = O.solve_one(ROSEN, [0.0], u0, O.ALG_NEWTON, g["abstol"], 1000)
    assert (st == O.ST_SUCCESS) == g["newton_converges"]
    u, st, it, r, _ = O.solve_one(ROSEN, [0.0], u0, O.ALG_NEWTON_BACKTRACK, g["abstol"], 1000)
    assert (st == O.ST_SUCCESS) == g["newton_backtracking_converges"]
    np.testing.assert_allclose(u, g["root"], rtol=0, atol=1e-9)
    u, st, it, r, _ = O.solve_one(ROSEN, [0.0], u0, O.ALG_TRUST_DOGLEG, g["abstol"], 1000)
    assert st == O.ST_SUCCESS
    np.testing.assert_allclose(u, g["root"], atol=1e-9)


def test_rosenbrock_gpu_example_inputs():
    # Sec. 3.3: u0 ~ U[0, 1)^10, plain Newton; root is the all-ones vector
    b = I.rosenbrock_batch(10, 256)
    u, st, it, r, _ = O.solve_batch(ROSEN, b.params, b.u0, O.ALG_NEWTON, 1e-8, 1000)
    ok = st == O.ST_SUCCESS
    assert ok.mean() > 0.95
    np.testing.assert_allclose(u[:, ok], 1.0, atol=1e-9)


# ---------------------------------------------------------------- general roots

def numpy_cubic_residual(A, b, u):
    return A @ u + u ** 3 - b


@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("n,w", [(3, 2.0), (8, 5.0), (16, 2.0)])
def test_cubic_dense_matches_minpack(alg, n, w):
    b = I.cubic_batch(n, 40, seed=0, config_id=1, b_half_width=w)
    u, st, it, r, _ = O.solve_batch(b.family, b.params, b.u0, alg)
    assert (st == O.ST_SUCCESS).all()
    for k in range(b.batch):
        A = b.params[: n * n, k].reshape(n, n)
        bb = b.params[n * n:, k]
        F = numpy_cubic_residual(A, bb, u[:, k])
        assert np.abs(F).max() <= 1e-10
        sol = scipy.optimize.root(lambda x: numpy_cubic_residual(A, bb, x), np.zeros(n),
                                  jac=lambda x: A + np.diag(3 * x ** 2), method="hybr",
                                  options={"xtol": 1e-14})
        # the root is unique (sym(A) > 0): any two solvers agree up to ||J^-1|| ||F||
        np.testing.assert_allclose(u[:, k], sol.x, rtol=0, atol=1e-9)


def test_cubic_generator_is_monotone():
    b = I.cubic_batch(8, 2000, config_id=1, b_half_width=5.0)
    A = b.params[:64].T.reshape(-1, 8, 8)
    assert np.linalg.eigvalsh(0.5 * (A + A.transpose(0, 2, 1)))[:, 0].min() > 0


@pytest.mark.parametrize("alg", ALGS)
def test_bratu_residual_invariant(alg):
    for n in (3, 9, 17, 33):
        bb = I.bratu_batch(n, 20, config_id=2)
        u, st, it, r, _ = O.solve_batch(BRATU, bb.params, bb.u0, alg)
        assert (st == O.ST_SUCCESS).all()
        for k in range(bb.batch):
            lam = bb.params[0, k]
            x = np.concatenate([[0.0], u[:, k], [0.0]])
            F = (x[:-2] - 2 * x[1:-1] + x[2:]) * (n + 1) ** 2 + lam * np.exp(x[1:-1])
            assert np.abs(F).max() <= 1e-10
            assert 0 < u[:, k].min() and u[:, k].max() < 0.7  # lower branch


# ---------------------------------------------------------------- Jacobian, LU

@pytest.mark.parametrize("family,n", [(CUBIC, 5), (BRATU, 7), (SQUARE, 4), (ROSEN, 6)])
def test_jacobian_matches_central_differences(family, n):
    rng = np.random.default_rng(3)
    E = I.n_params(family, n)
    p = rng.uniform(0.5, 2.0, size=max(E, 1))
    u = rng.uniform(-1, 1, size=n)
    J = O.jacobian(family, p, u)
    Jfd = np.empty((n, n))
    for j in range(n):
        h = 1e-6 * max(1.0, abs(u[j]))
        e = np.zeros(n)
        e[j] = h
        Jfd[:, j] = (O.residual(family, p, u + e) - O.residual(family, p, u - e)) / (2 * h)
    np.testing.assert_allclose(J, Jfd, rtol=1e-7, atol=1e-6)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 32, 64])
def test_lu_matches_lapack(n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n))
    LU, piv, info = O.lu_factor(A)
    assert info == 0
    lu_ref, piv_ref = scipy.linalg.lu_factor(A)
    np.testing.assert_array_equal(piv, piv_ref)
    np.testing.assert_allclose(LU, lu_ref, rtol=1e-12, atol=1e-12)
    # reconstruction P A = L U
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    PA = A.copy()
    for k in range(n):
        PA[[k, piv[k]]] = PA[[piv[k], k]]
    assert np.abs(PA - L @ U).max() <= 8 * n * np.finfo(float).eps * np.abs(A).max()
    x = O.lu_solve(LU, piv, A @ np.arange(1.0, n + 1))
    np.testing.assert_allclose(x, np.arange(1.0, n + 1), rtol=1e-9)


def cramer(A, b):
    d = np.linalg.det(A)
    out = np.empty(len(b))
    for i in range(len(b)):
        Ai = A.copy()
        Ai[:, i] = b
        out[i] = np.linalg.det(Ai) / d
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_lu_solve_cramer(n):
    rng = np.random.default_rng(10 + n)
    for _ in range(20):
        A = rng.normal(size=(n, n))
        b = rng.normal(size=n)
        LU, piv, info = O.lu_factor(A)
        np.testing.assert_allclose(O.lu_solve(LU, piv, b), cramer(A, b), rtol=1e-10, atol=1e-12)


def test_lu_pivot_is_argmax_with_lowest_index_tie():
    A = np.array([[1.0, 2.0], [-3.0, 1.0], [3.0, 0.0]])
    A = np.hstack([A, np.ones((3, 1))])
    LU, piv, info = O.lu_factor(A)
    assert piv[0] == 1  # |-3| = |3|: the lower index wins
    LU, piv, info = O.lu_factor(np.array([[0.0, 1.0], [0.0, 2.0]]))
    assert info == 1  # zero pivot column
    # comparisons with NaN are false: a NaN on the diagonal is kept as pivot -> singular
    LU, piv, info = O.lu_factor(np.array([[np.nan, 1.0], [1.0, 2.0]]))
    assert info == 1
    LU, piv, info = O.lu_factor(np.array([[1.0, 1.0], [np.nan, 2.0]]))
    assert piv[0] == 0
    LU, piv, info = O.lu_factor(np.array([[1.0, 2.0], [2.0, 4.0]]))
    assert info == 2


# ---------------------------------------------------------------- line search

def test_backtracking_hand_example():
    # F = u^2 - 1 from u0 = 0.1: Newton step 4.95; phi(1) and phi(1/2) violate
    # Armijo, alpha = 1/4 gives u = 1.3375 with phi = 0.311 < 0.49 (hand check)
    tr = O.solve_trace(SQUARE, [1.0], [0.1], O.ALG_NEWTON_BACKTRACK, 1e-12, 50)
    assert tr["alpha"][0] == 0.25 and tr["trials"][0] == 3
    assert tr["status"] == O.ST_SUCCESS and abs(tr["u"][0] - 1.0) <= 1e-12


@pytest.mark.parametrize("family,n,cfg", [(CUBIC, 8, 1), (ROSEN, 10, 0)])
def test_backtracking_armijo_holds_and_2alpha_fails(family, n, cfg):
    if family == CUBIC:
        b = I.cubic_batch(n, 30, config_id=cfg, b_half_width=5.0)
        cases = [(b.params[:, k], b.u0[:, k]) for k in range(b.batch)]
    else:
        u0 = np.ones(n)
        u0[0] = -1.2
        cases = [(np.zeros(1), u0)]
    checked = 0
    for p, u0 in cases:
        u = u0.copy()
        for _ in range(200):
            F = O.residual(family, p, u)
            if np.abs(F).max() <= 1e-10:
                break
            J = O.jacobian(family, p, u)
            dN = np.linalg.solve(J, -F)
            tr = O.solve_trace(family, p, u, O.ALG_NEWTON_BACKTRACK, 1e-10, 1)
            alpha = tr["alpha"][0]
            phi0, s = 0.5 * F @ F, F @ (J @ dN)
            phi = lambda a: 0.5 * np.sum(O.residual(family, p, u + a * dN) ** 2)
            assert phi(alpha) <= phi0 + 1e-4 * alpha * s + 1e-12 * abs(phi0)
            if alpha < 1.0:
                Fb = O.residual(family, p, u + 2 * alpha * dN)
                assert (not np.isfinite(Fb).all()) or phi(2 * alpha) > phi0 + 1e-4 * 2 * alpha * s
            assert alpha == 2.0 ** -(tr["trials"][0] - 1)
            u = tr["u"]
            checked += 1
    assert checked > 20


# ---------------------------------------------------------------- dogleg

def test_dogleg_hand_example_branches():
    # J = diag(1, 10), F = (1, 1): dN = (-1, -0.1); g = J^T F = (1, 10);
    # Cauchy point c = -(101/10001) g; ||c|| = 101^1.5/10001
    J = np.diag([1.0, 10.0])
    F = np.array([1.0, 1.0])
    dN = np.array([-1.0, -0.1])
    c = -(101.0 / 10001.0) * np.array([1.0, 10.0])
    norm_c = 101.0 ** 1.5 / 10001.0
    d, br = O.dogleg(J, F, dN, 2.0)
    assert br == 0 and np.array_equal(d, dN)
    d, br = O.dogleg(J, F, dN, 0.05)
    assert br == 1
    np.testing.assert_allclose(d, -0.05 * np.array([1.0, 10.0]) / math.sqrt(101.0), rtol=1e-15)
    d, br = O.dogleg(J, F, dN, 0.5)
    assert br == 2 and norm_c < 0.5
    tau = (d - c) @ (dN - c) / ((dN - c) @ (dN - c))
    assert 0 < tau < 1
    np.testing.assert_allclose(d, c + tau * (dN - c), rtol=1e-14, atol=1e-15)
    assert abs(np.linalg.norm(d) - 0.5) < 1e-15


def test_dogleg_minimises_model_along_path():
    rng = np.random.default_rng(5)
    for _ in range(50):
        n = rng.integers(2, 7)
        J = rng.normal(size=(n, n)) + 2 * np.eye(n)
        F = rng.normal(size=n)
        dN = np.linalg.solve(J, -F)
        g = J.T @ F
        c = -(g @ g) / ((J @ g) @ (J @ g)) * g
        Delta = rng.uniform(0.05, 1.5) * np.linalg.norm(dN)
        d, br = O.dogleg(J, F, dN, Delta)
        model = lambda s: 0.5 * np.sum((F + J @ s) ** 2)
        # brute force: the best point of the piecewise-linear path 0 -> c -> dN inside the ball
        ts = np.linspace(0, 1, 4001)
        path = [t * c for t in ts] + [c + t * (dN - c) for t in ts]
        # the first leg is a ray along -g: extend it to the boundary too
        path += [-(t * Delta / np.linalg.norm(g)) * g for t in ts]
        feas = [s for s in path if np.linalg.norm(s) <= Delta * (1 + 1e-12)]
        best = min(model(s) for s in feas)
        assert model(d) <= best + 1e-9 * (1 + abs(best))
        assert np.linalg.norm(d) <= Delta * (1 + 1e-14)
        if br != 0:
            assert abs(np.linalg.norm(d) - Delta) <= 1e-14 * Delta


def test_trust_region_radius_rules():
    b = I.cubic_batch(8, 40, config_id=1, b_half_width=5.0)
    seen = set()
    for k in range(b.batch):
        tr = O.solve_trace(CUBIC, b.params[:, k], b.u0[:, k], O.ALG_TRUST_DOGLEG, 1e-10, 50)
        assert tr["status"] == O.ST_SUCCESS
        rad, rho = tr["radius"], tr["rho"]
        assert rad[0] == 1.0
        for i in range(len(rad) - 1):
            if rho[i] > 0.75:
                expect = min(2 * rad[i], 1e3)
                seen.add("grow")
            elif rho[i] > 0:
                expect = rad[i]
                seen.add("keep")
            else:
                expect = 0.25 * rad[i]
                seen.add("shrink")
            assert rad[i + 1] == expect
        seen.update({f"branch{x}" for x in tr["branch"]})
    assert {"grow", "branch0", "branch1", "branch2"} <= seen


def test_trust_region_rho_is_one_on_linear_part():
    # a Bratu-free, cube-free case: diagonal cubic with b = 0 has u = 0 as the root;
    # the step from u0 with tiny |u0| is nearly linear so rho is within 1e-6 of 1
    A = (3.0 * np.eye(3)).reshape(-1)
    p = np.concatenate([A, np.zeros(3)])
    tr = O.solve_trace(CUBIC, p, np.full(3, 1e-3), O.ALG_TRUST_DOGLEG, 1e-300, 2)
    assert abs(tr["rho"][0] - 1.0) < 1e-5


# ---------------------------------------------------------------- statuses

def test_status_semantics():
    p = np.concatenate([(3.0 * np.eye(2)).reshape(-1), [1.0, np.nan]])
    for alg in ALGS:
        assert O.solve_one(CUBIC, p, np.zeros(2), alg)[1] == O.ST_NONFINITE
    p = np.concatenate([(3.0 * np.eye(2)).reshape(-1), [1.0, 2.0]])
    for alg in ALGS:
        u, st, it, r, _ = O.solve_one(CUBIC, p, np.zeros(2), alg, maxiters=2)
        assert st == O.ST_MAXITERS and it == 2 and r > 1e-10
    u, st, it, r, _ = O.solve_one(CUBIC, p, np.zeros(2), O.ALG_NEWTON, maxiters=0)
    assert st == O.ST_MAXITERS and it == 0 and r == 2.0
    root, *_ = O.solve_one(CUBIC, p, np.zeros(2), O.ALG_NEWTON)
    for alg in ALGS:
        u, st, it, r, _ = O.solve_one(CUBIC, p, root, alg, maxiters=0)
        assert st == O.ST_SUCCESS and it == 0
    u, st, it, r, _ = O.solve_one(ROSEN, [0.0], np.r_[-1.2, np.ones(9)], O.ALG_NEWTON, 1e-8, 1000)
    assert st == O.ST_NONFINITE and it == 9


def test_polish_reaches_rounding_floor():
    b = I.cubic_batch(8, 20, config_id=1, b_half_width=5.0)
    u, st, it, r, _ = O.solve_batch(b.family, b.params, b.u0, O.ALG_NEWTON)
    up = O.polish_batch(b.family, b.params, u)
    for k in range(b.batch):
        F = O.residual(CUBIC, b.params[:, k], up[:, k])
        assert np.abs(F).max() <= 4e-14


def test_threaded_batch_equals_serial():
    b = I.cubic_batch(8, 512, config_id=1, b_half_width=5.0)
    r1 = O.solve_batch(b.family, b.params, b.u0, O.ALG_TRUST_DOGLEG, threads=1)
    r4 = O.solve_batch(b.family, b.params, b.u0, O.ALG_TRUST_DOGLEG, threads=4)
    for a, c in zip(r1, r4):
        np.testing.assert_array_equal(a, c)


# ---------------------------------------------------------------- sensitivity (Sec. 2.3)

def test_adjoint_square_example_sec2_3():
    # g(u*) = sum u*^2 with u* = sqrt(p): dg/dp = 1 exactly (the example's gradient)
    g = golden("square_sec2_3.json")
    u, st, *_ = O.solve_one(SQUARE, g["p"], g["u0"], O.ALG_NEWTON, abstol=1e-14)
    grad, sing = O.adjoint(SQUARE, g["p"], u, 2.0 * u)
    assert not sing
    np.testing.assert_allclose(grad, g["dg_dtheta"], rtol=1e-15)
    # du*/dp = 1 / (2 sqrt(p)): cotangent e_i picks row i
    for i in range(2):
        e = np.zeros(2)
        e[i] = 1.0
        grad, _ = O.adjoint(SQUARE, g["p"], u, e)
        np.testing.assert_allclose(grad[i], 0.5 / np.sqrt(g["p"][i]), rtol=1e-15)
        assert grad[1 - i] == 0.0


@pytest.mark.parametrize("family,n", [(CUBIC, 3), (CUBIC, 6), (BRATU, 5), (SQUARE, 4),
                                      (CUBIC, 20), (BRATU, 64), (SQUARE, 40)])
def test_adjoint_matches_finite_differences(family, n):
    rng = np.random.default_rng(7)
    if family == CUBIC:
        b = I.cubic_batch(n, 1, config_id=8)
    elif family == BRATU:
        b = I.bratu_batch(n, 1, config_id=8)
    else:
        b = I.square_batch(n, 1)
    p = b.params[:, 0].copy()
    u, st, *_ = O.solve_one(family, p, b.u0[:, 0], O.ALG_NEWTON, abstol=1e-14)
    w = rng.normal(size=n)
    grad, sing = O.adjoint(family, p, u, w)
    assert not sing
    for e in range(p.size):
        # larger systems reach their root to about n eps cond(J): a wider
        # difference step keeps that round-off below the tolerance
        h = (1e-6 if n <= 8 else 1e-4) * max(1.0, abs(p[e]))
        pp, pm = p.copy(), p.copy()
        pp[e] += h
        pm[e] -= h
        up, *_ = O.solve_one(family, pp, u, O.ALG_NEWTON, abstol=1e-15)
        um, *_ = O.solve_one(family, pm, u, O.ALG_NEWTON, abstol=1e-15)
        fd = w @ (up - um) / (2 * h)
        assert abs(grad[e] - fd) <= 1e-6 * (1 + abs(fd)), (e, grad[e], fd)
