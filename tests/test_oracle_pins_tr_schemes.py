"""Pins of the oracle's NocedalWright trust-region radius update (Sec. 2.2.2,
Tab. 3; Algorithm 4.1 of Nocedal & Wright, the paper's reference for it)
against hand-derived one-dimensional passes, where every quantity is an
exact rational (F is a polynomial, the dogleg step in 1-D is the Newton
step or +-Delta):

  F(u) = a u + u^3 - b (the cubic family with n = 1), J = a + 3u^2,
  rho = (F0^2 - F1^2) / (F0^2 - (F0 + J0 d)^2).

The rules: shrink to Delta/4 when rho < 1/4; double (capped) when
rho > 3/4 and the step reached the boundary; otherwise keep Delta; accept
the step when rho > eta = 1e-4.  The "Simple" reading, for contrast,
accepts when rho > 0, doubles when rho > 3/4 wherever the step ended, and
shrinks only on rejection.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O
from paper_2403_16341_gb300 import inputs as I

CUBIC = 0
NW, SIMPLE = O.ALG_TRUST_DOGLEG_NW, O.ALG_TRUST_DOGLEG


def trace(a, b, u0, alg, k=1):
    return O.solve_trace(CUBIC, [a, b], [u0], alg, abstol=0.0, maxiters=k + 1)


def test_interior_step_good_model_keeps_radius():
    # a = 1, b = 0, u0 = 2: F0 = 10, J0 = 13, dN = -10/13 inside Delta0 = 1
    # (branch N); u1 = 16/13, F1 = 16/13 + 4096/2197 = 6800/2197, pred = 100
    F1 = Fr(6800, 2197)
    rho = (100 - F1 * F1) / 100  # 0.904...
    r_nw = trace(1.0, 0.0, 2.0, NW)
    r_s = trace(1.0, 0.0, 2.0, SIMPLE)
    for r in (r_nw, r_s):
        assert r["branch"][0] == 0
        assert abs(r["rho"][0] - float(rho)) < 1e-15
    assert r_nw["radius"][1] == 1.0   # interior step: no growth
    assert r_s["radius"][1] == 2.0    # Simple grows wherever the step ended


def test_poor_model_accepts_and_shrinks():
    # a = -1, b = 1, u0 = 1: F0 = -1, J0 = 2, dN = 1/2 (branch N), u1 = 3/2,
    # F1 = 7/8, pred = 1, rho = 1 - 49/64 = 15/64 in (eta, 1/4)
    r_nw = trace(-1.0, 1.0, 1.0, NW)
    r_s = trace(-1.0, 1.0, 1.0, SIMPLE)
    for r in (r_nw, r_s):
        assert r["branch"][0] == 0
        assert r["rho"][0] == 15 / 64
    assert r_nw["radius"][1] == 0.25  # accepted, but the radius shrinks
    assert r_s["radius"][1] == 1.0
    # both accepted the step: the second pass starts from u1 = 3/2, whose
    # Newton step is -F1 / J1 = -(7/8) / (23/4) = -7/46
    u_nw = O.solve_one(CUBIC, [-1.0, 1.0], [1.0], NW, abstol=0.0, maxiters=1)[0]
    assert u_nw[0] == 1.5


def test_fair_model_keeps_radius():
    # a = -1, b = -1, u0 = 1: F0 = 1, J0 = 2, dN = -1/2 (branch N), u1 = 1/2,
    # F1 = 5/8, pred = 1, rho = 1 - 25/64 = 39/64 in [1/4, 3/4]: keep Delta
    # a = 1/2, b = 1, u0 = 1/2: F0 = -5/8, J0 = 5/4, dN = 1/2, u1 = 1, F1 = 1/2,
    # pred = 25/64, rho = (25/64 - 16/64) / (25/64) = 9/25, also kept
    for alg in (NW, SIMPLE):
        r = trace(-1.0, -1.0, 1.0, alg)
        assert r["branch"][0] == 0 and r["rho"][0] == 39 / 64
        assert r["radius"][1] == 1.0
        r = trace(0.5, 1.0, 0.5, alg)
        assert r["branch"][0] == 0 and abs(r["rho"][0] - 9 / 25) < 1e-15
        assert r["radius"][1] == 1.0


def test_bad_step_is_rejected_and_shrinks():
    # a = -1, b = 1, u0 = 3/5: F0 = -173/125, J0 = 2/25, dN = 17.3 > Delta0 = 1;
    # in 1-D the Cauchy point is dN, so branch C takes d = +1 (g = J0 F0 < 0);
    # u1 = 8/5, F1 = 187/125: ared = (173^2 - 187^2)/125^2 < 0,
    # pred = (173^2 - 163^2)/125^2, rho = -5040/3360 = -3/2
    for alg in (NW, SIMPLE):
        r = trace(-1.0, 1.0, 0.6, alg)
        assert r["branch"][0] == 1
        assert abs(r["rho"][0] - (-1.5)) < 1e-12
        assert r["radius"][1] == 0.25
        u = O.solve_one(CUBIC, [-1.0, 1.0], [0.6], alg, abstol=0.0, maxiters=1)[0]
        assert u[0] == 0.6  # rejected: u unchanged


def test_radius_changes_follow_the_rules_on_a_long_walk():
    # u^2 = 1e8 from u0 = 1: a long walk with growing, kept and shrunk radii;
    # every change seen in the record is one the rules allow
    p = 1e8
    r = O.solve_trace(2, [p], [1.0], NW, abstol=1e-6, maxiters=60)
    assert r["status"] == O.ST_SUCCESS
    rad = r["radius"]
    assert rad.max() <= 1e3
    grew = [k for k in range(1, rad.size) if rad[k] > rad[k - 1]]
    for k in grew:
        assert rad[k] == min(2 * rad[k - 1], 1e3)
        assert r["branch"][k - 1] != 0 and r["rho"][k - 1] > 0.75
    shrunk = [k for k in range(1, rad.size) if rad[k] < rad[k - 1]]
    for k in shrunk:
        assert rad[k] == 0.25 * rad[k - 1] and r["rho"][k - 1] < 0.25


@pytest.mark.parametrize("family,n", [(0, 6), (1, 5), (2, 4), (3, 8)])
def test_nocedal_wright_reaches_pinned_roots(family, n):
    if family == 0:
        b = I.cubic_batch(n, 64, config_id=2)
    elif family == 1:
        b = I.bratu_batch(n, 64)
    elif family == 2:
        b = I.square_batch(n, 64)
    else:
        b = I.rosenbrock_batch(n, 64, seed=0)
    # NocedalWright also shrinks after accepted steps with rho < 1/4: on the
    # curved Rosenbrock valley it needs up to 140 passes where Simple needs 80
    u, st, it, r, _ = O.solve_batch(b.family, b.params, b.u0, NW, abstol=1e-10, maxiters=300)
    assert (st == O.ST_SUCCESS).mean() > 0.95
    ok = st == O.ST_SUCCESS
    if family == 2:
        np.testing.assert_allclose(np.abs(u[:, ok]), np.sqrt(b.params[:, ok]), atol=1e-10)
    elif family == 3:
        np.testing.assert_allclose(u[:, ok], 1.0, atol=1e-8)
    else:
        # the Simple scheme's roots (themselves pinned to Cardano, MINPACK and
        # bisection) are the same roots
        u2, st2, _, _, _ = O.solve_batch(b.family, b.params, b.u0, SIMPLE, abstol=1e-10,
                                         maxiters=300)
        both = ok & (st2 == O.ST_SUCCESS)
        np.testing.assert_allclose(u[:, both], u2[:, both], rtol=1e-9, atol=1e-10)
