"""GPU parity of the warp-tiled solver (one instance per 8/16/32-lane
segment, n <= 32) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from paper_2403_16341_gb300 import inputs as I
from tests.parity import FP64_TOL, MIXED_TOL, check_parity, gpu_solve, oracle_solve, rel_err

pytestmark = pytest.mark.gpu

NEWTON, LS, TR = 0, 1, 2
MIXED, TILE_THREAD, TILE_WARP = 1 << 8, 1 << 10, 1 << 11


@pytest.fixture(scope="module")
def solver():
    import paper_2403_16341_gb300 as nls
    s = nls.Solver(0)
    yield s
    s.close()


def make(family, n, B, cfg=2):
    if family == I.FAMILY_CUBIC:
        return I.cubic_batch(n, B, config_id=cfg)
    if family == I.FAMILY_BRATU:
        return I.bratu_batch(n, B, config_id=cfg)
    if family == I.FAMILY_SQUARE:
        return I.square_batch(n, B)
    return I.rosenbrock_batch(n, B)


@pytest.mark.parametrize("family", [I.FAMILY_CUBIC, I.FAMILY_BRATU, I.FAMILY_SQUARE,
                                    I.FAMILY_ROSENBROCK])
@pytest.mark.parametrize("n", [9, 13, 16, 17, 25, 32])
@pytest.mark.parametrize("alg", [NEWTON, LS, TR])
@pytest.mark.parametrize("mixed", [False, True])
def test_warp_parity(solver, family, n, alg, mixed):
    b = make(family, n, 67)
    maxiters = 300 if family == I.FAMILY_ROSENBROCK else 50
    g = gpu_solve(solver, b, alg | (MIXED if mixed else 0), maxiters=maxiters)
    o = oracle_solve(b, alg, maxiters=maxiters)
    # plain Newton on Rosenbrock from U[0,1)^n is rounding-chaotic for n >= 13
    chaotic = family == I.FAMILY_ROSENBROCK and alg == NEWTON and n >= 13
    check_parity(b, g, o, mixed, rule="chaotic" if chaotic else "exact", alg=alg,
                 maxiters=maxiters)
    if family == I.FAMILY_ROSENBROCK:
        ok = g["status"] == 0
        np.testing.assert_allclose(g["u"][:, ok], 1.0, atol=1e-9)


@pytest.mark.parametrize("n", [2, 3, 5, 8])
@pytest.mark.parametrize("alg", [NEWTON, LS, TR])
@pytest.mark.parametrize("mixed", [False, True])
def test_warp_matches_thread_tiling(solver, n, alg, mixed):
    b = I.cubic_batch(n, 301, config_id=1, b_half_width=5.0)
    m = MIXED if mixed else 0
    gt = gpu_solve(solver, b, alg | m | TILE_THREAD)
    gw = gpu_solve(solver, b, alg | m | TILE_WARP)
    np.testing.assert_array_equal(gw["status"], gt["status"])
    assert rel_err(gw["u"], gt["u"]).max() <= (MIXED_TOL if mixed else FP64_TOL)
    o = oracle_solve(b, alg)
    check_parity(b, gw, o, mixed)


def test_rosenbrock_gpu_example_sec3_4(solver):
    # 1024 ten-dimensional generalized Rosenbrock problems, u0 ~ U[0, 1)^10, plain Newton
    b = I.rosenbrock_batch(10, 1024)
    g = gpu_solve(solver, b, NEWTON, abstol=1e-8, maxiters=1000)
    o = oracle_solve(b, NEWTON, abstol=1e-8, maxiters=1000)
    np.testing.assert_array_equal(g["status"], o["status"])
    ok = g["status"] == 0
    assert ok.mean() > 0.95
    np.testing.assert_allclose(g["u"][:, ok], 1.0, atol=1e-9)


def test_warp_persistent_and_static_agree_bitwise(solver):
    import paper_2403_16341_gb300 as nls
    for n in (12, 30):
        b = I.cubic_batch(n, 1500, config_id=4)
        runs = []
        for persistent in (0, 1):
            solver.set_option(nls.NLS_OPT_PERSISTENT, persistent)
            runs.append(gpu_solve(solver, b, TR | MIXED))
        solver.set_option(nls.NLS_OPT_PERSISTENT, 1)
        for key in ("u", "status", "iters", "resid", "nfev"):
            np.testing.assert_array_equal(runs[1][key], runs[0][key])


def test_warp_singular_and_nan(solver):
    sq = I.Batch(I.FAMILY_SQUARE, 12, np.full((12, 3), 2.0), np.zeros((12, 3)))
    g = gpu_solve(solver, sq, NEWTON)
    assert (g["status"] == O.ST_SINGULAR).all() and (g["iters"] == 1).all()
    b = I.cubic_batch(20, 5, config_id=3)
    b.params[7, 2] = np.nan
    g = gpu_solve(solver, b, LS)
    assert g["status"][2] == O.ST_NONFINITE and (np.delete(g["status"], 2) == 0).all()
