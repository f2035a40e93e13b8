"""GPU parity of the Potra-Ptak (Eq. 4), Halley (Eq. 3), Broyden and modified
Broyden (Tab. 1) kernels against the FP64 oracle, through the C ABI.

Tolerances are those of the Newton kernels (1e-9 FP64, 1e-8 mixed,
relative to max(1, ||u*||_inf), or the conditioning bound).  Statuses
follow the rule of each case (status_rule below, tests/parity.py):
Halley's statuses are compared exactly; the local methods (Potra-Ptak and
the two Broydens, which can cycle or diverge) by their solved sets, which
must equal the oracle's in FP64 apart from instances the oracle ends in
its last five passes and instances whose outcome rounding decides (shown
by the oracle's own per-pass jitter); Rosenbrock from U[0,1)^n is
rounding-chaotic for every method.  The GPU keeps
B^-1 by Sherman-Morrison where the oracle refactors B, so Broyden is
compared by outcome and root, not by bits."""
import numpy as np
import pytest

import oracle as O
from paper_2403_16341_gb300 import inputs as I
from tests.parity import check_parity, gpu_solve, late_instances, oracle_solve

pytestmark = pytest.mark.gpu

PP, HALLEY, BROYDEN, MOD_BROYDEN = 4, 5, 6, 7
MIXED, ANALYTIC = 1 << 8, 1 << 9
TILE_WARP, TILE_CTA = 1 << 11, 1 << 12
NEXT4 = (PP, HALLEY, BROYDEN, MOD_BROYDEN)


@pytest.fixture(scope="module")
def solver():
    import paper_2403_16341_gb300 as nls
    s = nls.Solver(0)
    yield s
    s.close()


def family_batch(family, n, B):
    if family == I.FAMILY_CUBIC:
        return I.cubic_batch(n, B, config_id=2)
    if family == I.FAMILY_BRATU:
        return I.bratu_batch(n, B)
    if family == I.FAMILY_SQUARE:
        return I.square_batch(n, B)
    return I.rosenbrock_batch(n, B, seed=0)


def status_rule(family, alg):
    """The status rule of check_parity for one case: the generalized
    Rosenbrock function from U[0,1)^n is rounding-chaotic for every method
    here; the local methods (Potra-Ptak, Broyden, modified Broyden) are
    compared by their solved sets; Halley exactly."""
    if family == I.FAMILY_ROSENBROCK:
        return "chaotic"
    if alg in (PP, BROYDEN, MOD_BROYDEN):
        return "success_set"
    return "exact"


@pytest.mark.parametrize("family", [I.FAMILY_CUBIC, I.FAMILY_BRATU, I.FAMILY_SQUARE,
                                    I.FAMILY_ROSENBROCK])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("alg", NEXT4)
@pytest.mark.parametrize("mixed", [False, True])
def test_families_all_sizes(solver, family, n, alg, mixed):
    if family == I.FAMILY_BRATU and n == 1:
        n = 2
    b = family_batch(family, n, 97)
    g = gpu_solve(solver, b, alg | (MIXED if mixed else 0))
    o = oracle_solve(b, alg)
    check_parity(b, g, o, mixed, rule=status_rule(family, alg), alg=alg)


@pytest.mark.parametrize("alg", [HALLEY, MOD_BROYDEN, PP])
@pytest.mark.parametrize("mixed", [False, True])
def test_cubic_n8_parity_ragged(solver, alg, mixed):
    # the cubic n = 8 workload (b ~ U[-5, 5]^8), several warps and a ragged tail
    b = I.cubic_batch(8, 4099, config_id=1, b_half_width=5.0)
    g = gpu_solve(solver, b, alg | (MIXED if mixed else 0))
    o = oracle_solve(b, alg)
    err = check_parity(b, g, o, mixed, rule=status_rule(b.family, alg), alg=alg)
    if alg != PP:
        assert g["solved"] == b.batch
    if not mixed and alg != PP:
        # FP64 mode follows the oracle's iteration count almost everywhere
        assert (g["iters"] == o["iters"]).mean() > 0.97
    print(f"alg {alg} mixed {mixed}: max rel err {err.max():.2e}, iters gpu "
          f"{g['iters'].mean():.2f} oracle {o['iters'].mean():.2f}")


@pytest.mark.parametrize("alg", [PP, HALLEY, MOD_BROYDEN, BROYDEN])
def test_residual_counts(solver, alg):
    b = I.cubic_batch(3, 500, config_id=2)
    g = gpu_solve(solver, b, alg)
    o = oracle_solve(b, alg)
    same = (g["status"] == 0) & (o["status"] == 0) & (g["iters"] == o["iters"])
    assert same.mean() > 0.9
    per_pass = 2 if alg == PP else 1
    np.testing.assert_array_equal(g["nfev"][same], 1 + per_pass * g["iters"][same])
    np.testing.assert_array_equal(g["nfev"][same], o["nfev"][same])


def test_halley_zero_denominator(solver):
    # component 0 starts at its root: a_0 = 0 = b_0, the step component is 0
    b = I.Batch(I.FAMILY_SQUARE, 2, np.array([[4.0], [2.0]]), np.array([[2.0], [1.0]]))
    g = gpu_solve(solver, b, HALLEY, abstol=1e-14)
    assert g["status"][0] == 0 and g["u"][0, 0] == 2.0
    assert abs(g["u"][1, 0] - np.sqrt(2.0)) < 1e-15


@pytest.mark.parametrize("mixed", [False, True])
def test_singular_cases(solver, mixed):
    # u0 = 0 on the square family: J = diag(2u) = 0 -> SINGULAR at pass 1 for
    # the Jacobian methods; Broyden from B_0 = I on u^2 = 3 from 3 steps to -3
    # where F is unchanged: df = 0 makes the updated B singular -> SINGULAR at
    # pass 2 (both sides, exactly: every value is an integer)
    m = MIXED if mixed else 0
    z = I.Batch(I.FAMILY_SQUARE, 2, np.array([[2.0], [3.0]]), np.zeros((2, 1)))
    for alg in (PP, HALLEY, MOD_BROYDEN):
        g = gpu_solve(solver, z, alg | m)
        assert g["status"][0] == O.ST_SINGULAR and g["iters"][0] == 1
    s = I.Batch(I.FAMILY_SQUARE, 1, np.array([[3.0]]), np.array([[3.0]]))
    g = gpu_solve(solver, s, BROYDEN | m)
    o = oracle_solve(s, BROYDEN)
    assert o["status"][0] == O.ST_SINGULAR and o["iters"][0] == 2
    assert g["status"][0] == O.ST_SINGULAR and g["iters"][0] == 2


def test_edge_sizes(solver):
    import paper_2403_16341_gb300 as nls
    import torch
    # empty batch; maxiters 0; a ragged single warp
    for alg in NEXT4:
        b = I.cubic_batch(4, 33, config_id=2)
        g = gpu_solve(solver, b, alg, maxiters=0)
        assert (g["status"] == O.ST_MAXITERS).all() and (g["iters"] == 0).all()
        u0 = torch.zeros((4, 0), dtype=torch.float64, device="cuda")
        p = torch.zeros((20, 0), dtype=torch.float64, device="cuda")
        out = nls.solve(I.FAMILY_CUBIC, p, u0, alg, 1e-10, 50, solver)
        assert out[-1] == 0


def test_unsupported_combinations(solver):
    import paper_2403_16341_gb300 as nls
    import torch
    b = I.cubic_batch(4, 8, config_id=2)
    p = torch.from_numpy(b.params).cuda()
    u = torch.from_numpy(b.u0).cuda()
    for alg in NEXT4:
        with pytest.raises(nls.NlsError) as e:
            nls.solve(I.FAMILY_CUBIC, p, u, alg | ANALYTIC, 1e-10, 50, solver)
        assert e.value.code == nls.NLS_E_UNSUPPORTED
    # a forced tiling that cannot hold n
    b33 = I.cubic_batch(33, 8, config_id=2)
    p33, u33 = torch.from_numpy(b33.params).cuda(), torch.from_numpy(b33.u0).cuda()
    for bad in (HALLEY | nls.NLS_TILE_WARP, HALLEY | nls.NLS_TILE_THREAD):
        with pytest.raises(nls.NlsError) as e:
            nls.solve(I.FAMILY_CUBIC, p33, u33, bad, 1e-10, 50, solver)
        assert e.value.code == nls.NLS_E_UNSUPPORTED
    with pytest.raises(nls.NlsError) as e:
        nls.solve(I.FAMILY_CUBIC, p, u, 8, 1e-10, 50, solver)
    assert e.value.code == nls.NLS_E_INVALID


@pytest.mark.parametrize("alg", [HALLEY, MOD_BROYDEN, PP, BROYDEN])
def test_full_size(solver, alg):
    # the cubic n = 8, 2^20 workload in the launch mode the benchmark uses
    # (autotuned): the solved set against the oracle's over the whole batch
    # (Halley: every instance solved; the local methods: the success_set
    # rule), the roots on a sample of 300 instances
    import torch
    b = I.workload_cubic_n8()
    o = oracle_solve(b, alg, threads=16)
    ok_o = o["status"] == 0
    for mixed in (False, True):
        late = late_instances(o, margin=10 if mixed else 5)
        a = alg | (MIXED if mixed else 0)
        p = torch.from_numpy(b.params).cuda()
        u0 = torch.from_numpy(b.u0).cuda()
        solver.autotune(b.family, p, u0.clone(), a, 1e-10, 50)
        g = gpu_solve(solver, b, a)
        ok_g = g["status"] == 0
        if alg == HALLEY:
            assert g["solved"] == b.batch and ok_o.all()
        else:
            bad = (ok_o & ~ok_g) if mixed else (ok_o != ok_g)
            sel = np.nonzero(bad & ~late)[0]
            print(f"alg {alg} mixed {mixed}: solved gpu {int(ok_g.sum())} oracle {int(ok_o.sum())}, "
                  f"{int((bad & late).sum())} late differences, {sel.size} others")
            if sel.size:
                # every other difference must be judged by the rule on its own
                sub = I.Batch(b.family, b.n, np.ascontiguousarray(b.params[:, sel]),
                              np.ascontiguousarray(b.u0[:, sel]))
                gs = {k: (v[..., sel] if isinstance(v, np.ndarray) else v) for k, v in g.items()}
                gs["solved"] = int((gs["status"] == 0).sum())
                os_ = {k: v[..., sel] for k, v in o.items()}
                check_parity(sub, gs, os_, mixed, rule="success_set", alg=alg)
        rng = np.random.default_rng(7)
        idx = np.sort(rng.choice(b.batch, 300, replace=False))
        sub = I.Batch(b.family, b.n, np.ascontiguousarray(b.params[:, idx]), np.ascontiguousarray(b.u0[:, idx]))
        gs = {k: (v[..., idx] if isinstance(v, np.ndarray) else v) for k, v in g.items()}
        gs["solved"] = int((gs["status"] == 0).sum())
        os_ = {k: v[..., idx] for k, v in o.items()}
        check_parity(sub, gs, os_, mixed, rule=status_rule(b.family, alg), alg=alg)


@pytest.mark.parametrize("family", [I.FAMILY_CUBIC, I.FAMILY_BRATU, I.FAMILY_SQUARE,
                                    I.FAMILY_ROSENBROCK])
@pytest.mark.parametrize("n", [9, 12, 16, 17, 24, 32])
@pytest.mark.parametrize("alg", NEXT4)
@pytest.mark.parametrize("mixed", [False, True])
def test_warp_tiling(solver, family, n, alg, mixed):
    # 8 < n <= 32: one instance per segment of 16 or 32 lanes; Rosenbrock from
    # U[0, 1)^n is rounding-decided for every method here (Potra-Ptak's starts
    # sit at the edge of its basin already at n = 9, 76% solved at n = 12)
    b = family_batch(family, n, 67)
    g = gpu_solve(solver, b, alg | (MIXED if mixed else 0))
    o = oracle_solve(b, alg)
    check_parity(b, g, o, mixed, rule=status_rule(family, alg), alg=alg)


@pytest.mark.parametrize("alg", NEXT4)
def test_warp_tiling_forced_small_n(solver, alg):
    # the warp kernels also hold n <= 8 when asked to (segments of 16 lanes)
    b = I.cubic_batch(5, 131, config_id=2)
    g = gpu_solve(solver, b, alg | TILE_WARP)
    o = oracle_solve(b, alg)
    check_parity(b, g, o, False, rule=status_rule(b.family, alg), alg=alg)


@pytest.mark.parametrize("family", [I.FAMILY_CUBIC, I.FAMILY_BRATU, I.FAMILY_SQUARE])
@pytest.mark.parametrize("n", [33, 40, 64, 65, 100, 128])
@pytest.mark.parametrize("alg", NEXT4)
@pytest.mark.parametrize("mixed", [False, True])
def test_cta_tiling(solver, family, n, alg, mixed):
    # 32 < n <= 128: one instance per CTA (register tiles R = 4 or 8); the
    # oracle solves every instance with Potra-Ptak, Halley and modified
    # Broyden and none with Broyden from B_0 = I
    b = family_batch(family, n, 37)
    g = gpu_solve(solver, b, alg | (MIXED if mixed else 0))
    o = oracle_solve(b, alg)
    check_parity(b, g, o, mixed, rule=status_rule(family, alg), alg=alg)
    if alg != BROYDEN:
        assert g["solved"] == b.batch


@pytest.mark.parametrize("alg", NEXT4)
def test_cta_tiling_forced_small_n(solver, alg):
    # the CTA kernels also hold small n when asked to
    b = I.cubic_batch(12, 45, config_id=2)
    g = gpu_solve(solver, b, alg | TILE_CTA)
    o = oracle_solve(b, alg)
    check_parity(b, g, o, False, rule=status_rule(b.family, alg), alg=alg)

