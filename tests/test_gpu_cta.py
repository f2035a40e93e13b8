"""GPU parity of the CTA-tiled solver (one instance per 256-thread CTA,
register-tiled LU, 32 < n <= 128) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from paper_2403_16341_gb300 import inputs as I
from tests.parity import FP64_TOL, MIXED_TOL, check_parity, gpu_solve, oracle_solve, rel_err

pytestmark = pytest.mark.gpu

NEWTON, LS, TR = 0, 1, 2
MIXED, TILE_WARP, TILE_CTA = 1 << 8, 1 << 11, 1 << 12
REFINE = 1 << 14


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
@pytest.mark.parametrize("n", [33, 47, 64, 65, 100, 128])
@pytest.mark.parametrize("alg", [NEWTON, LS, TR])
@pytest.mark.parametrize("mixed", [False, True])
def test_cta_parity(solver, family, n, alg, mixed):
    if family == I.FAMILY_ROSENBROCK and alg == NEWTON:
        pytest.skip("plain Newton on Rosenbrock from U[0,1)^n, n > 32, is rounding-chaotic")
    B = 23
    b = make(family, n, B)
    maxiters = 400 if family == I.FAMILY_ROSENBROCK else 50
    g = gpu_solve(solver, b, alg | (MIXED if mixed else 0), maxiters=maxiters)
    o = oracle_solve(b, alg, maxiters=maxiters)
    check_parity(b, g, o, mixed)


@pytest.mark.parametrize("n", [9, 20, 32])
@pytest.mark.parametrize("alg", [NEWTON, LS, TR])
@pytest.mark.parametrize("mixed", [False, True])
def test_cta_matches_warp_tiling(solver, n, alg, mixed):
    for family in (I.FAMILY_CUBIC, I.FAMILY_BRATU):
        b = make(family, n, 41)
        m = MIXED if mixed else 0
        gw = gpu_solve(solver, b, alg | m | TILE_WARP)
        gc = gpu_solve(solver, b, alg | m | TILE_CTA)
        np.testing.assert_array_equal(gc["status"], gw["status"])
        assert rel_err(gc["u"], gw["u"]).max() <= (MIXED_TOL if mixed else FP64_TOL)


@pytest.mark.parametrize("mixed", [False, True])
def test_bratu_large_full_size_sampled(solver, mixed):
    # 16,384 Bratu instances with n uniform in 64..128, trust-region dogleg,
    # FP32 LU with FP64 residual (mixed) or FP64 LU; the oracle solves a sample
    batches = I.workload_bratu_large()
    assert sum(b.batch for b in batches) == 16384
    rng = np.random.default_rng(1)
    checked = 0
    for b in batches:
        g = gpu_solve(solver, b, TR | (MIXED if mixed else 0))
        assert g["solved"] == b.batch and (g["resid"] <= 1e-10).all()
        if rng.random() < 0.2 or b.n in (64, 128):
            idx = np.sort(rng.choice(b.batch, min(4, b.batch), replace=False))
            sub = I.Batch(b.family, b.n, b.params[:, idx], b.u0[:, idx])
            gs = {k: (v[:, idx] if k == "u" else v[idx]) for k, v in g.items() if k != "solved"}
            gs["solved"] = int((gs["status"] == 0).sum())
            check_parity(sub, gs, oracle_solve(sub, TR), mixed)
            checked += idx.size
    assert checked >= 40


@pytest.mark.parametrize("family", [I.FAMILY_CUBIC, I.FAMILY_BRATU, I.FAMILY_SQUARE,
                                    I.FAMILY_ROSENBROCK])
@pytest.mark.parametrize("n", [5, 33, 64, 100, 128])
@pytest.mark.parametrize("alg", [NEWTON, LS, TR])
def test_refined_mixed_parity(solver, family, n, alg):
    # FP32 LU with two steps of classical iterative refinement per Newton
    # step (r = -F - J dN in FP64, re-solved with the FP32 factors): the
    # Newton steps are FP64-accurate, so the roots meet the FP64 gate and the
    # pass counts follow the FP64 oracle's
    if family == I.FAMILY_ROSENBROCK and n > 16:
        n = 16  # the Rosenbrock conditioning grows like 2^n
    b = make(family, n, 61)
    g = gpu_solve(solver, b, alg | MIXED | REFINE)
    o = oracle_solve(b, alg)
    # statuses: every instance the oracle solves is solved (the mixed rule);
    # Rosenbrock from U[0,1)^n keeps its chaotic rule
    rule = "chaotic" if family == I.FAMILY_ROSENBROCK else "exact"
    err = check_parity(b, g, o, mixed=True, rule=rule, alg=alg)
    both = (g["status"] == 0) & (o["status"] == 0)
    if family != I.FAMILY_ROSENBROCK:
        assert err.max() <= FP64_TOL
        assert (g["iters"][both] == o["iters"][both]).mean() >= 0.95


def test_refined_mixed_bratu_large_sampled(solver):
    # the Bratu n = 64..128 configuration with refinement: every instance
    # solved, the sampled roots within the FP64 gate, and the mean pass count
    # of the FP64-LU kernel (the refined steps are FP64-accurate)
    batches = I.workload_bratu_large()
    rng = np.random.default_rng(2)
    checked = 0
    for b in batches[::4]:
        g = gpu_solve(solver, b, TR | MIXED | REFINE)
        g64 = gpu_solve(solver, b, TR)
        assert g["solved"] == b.batch and (g["resid"] <= 1e-10).all()
        assert abs(g["iters"].mean() - g64["iters"].mean()) <= 0.05
        idx = np.sort(rng.choice(b.batch, min(4, b.batch), replace=False))
        sub = I.Batch(b.family, b.n, b.params[:, idx], b.u0[:, idx])
        gs = {k: (v[:, idx] if k == "u" else v[idx]) for k, v in g.items() if k != "solved"}
        gs["solved"] = int((gs["status"] == 0).sum())
        err = check_parity(sub, gs, oracle_solve(sub, TR), False)
        assert err.max() <= FP64_TOL
        checked += idx.size
    assert checked >= 40


def test_refine_flag_combinations(solver):
    import paper_2403_16341_gb300 as nls
    import torch
    b = I.cubic_batch(40, 8, config_id=2)
    p = torch.from_numpy(np.ascontiguousarray(b.params)).cuda()
    u = torch.from_numpy(np.ascontiguousarray(b.u0)).cuda()
    for alg in (LS | REFINE, LS | MIXED | REFINE | TILE_WARP, 4 | MIXED | REFINE, 3 | MIXED | REFINE):
        with pytest.raises(nls.NlsError) as e:
            solver.submit(b.family, p, u, alg)
        assert e.value.code == nls.NLS_E_UNSUPPORTED
    with pytest.raises(nls.NlsError) as e:
        solver.autotune(b.family, p, u, LS | MIXED | REFINE)
    assert e.value.code == nls.NLS_E_UNSUPPORTED


def test_cta_singular_nan_and_maxiters(solver):
    sq = I.Batch(I.FAMILY_SQUARE, 70, np.full((70, 2), 2.0), np.zeros((70, 2)))
    g = gpu_solve(solver, sq, NEWTON)
    assert (g["status"] == O.ST_SINGULAR).all() and (g["iters"] == 1).all()
    b = I.bratu_batch(90, 4, config_id=3)
    b.params[0, 1] = np.nan
    g = gpu_solve(solver, b, TR)
    assert g["status"][1] == O.ST_NONFINITE and (np.delete(g["status"], 1) == 0).all()
    g = gpu_solve(solver, I.bratu_batch(90, 3, config_id=3), LS, maxiters=1)
    assert (g["status"] == O.ST_MAXITERS).all() and (g["iters"] == 1).all()
