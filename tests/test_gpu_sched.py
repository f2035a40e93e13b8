"""Scheduler and autotuner: requests flushed together run as one CUDA-graph
launch of concurrent persistent kernels; each result equals the same request
solved alone; the autotuner's choices are valid and persist."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2403_16341_gb300 import inputs as I
from tests.parity import check_parity, gpu_solve, oracle_solve

pytestmark = pytest.mark.gpu

NEWTON, LS, TR = 0, 1, 2
MIXED = 1 << 8


@pytest.fixture(scope="module")
def solver():
    import paper_2403_16341_gb300 as nls
    s = nls.Solver(0)
    yield s
    s.close()


def submit_all(solver, batches, alg):
    """Every batch in one flush; `alg` is one algorithm word for all of them
    or a list with one per batch (precision may differ between buckets)."""
    import torch
    algs = list(alg) if isinstance(alg, (list, tuple)) else [alg] * len(batches)
    held, reqs = [], []
    for b, alg in zip(batches, algs):
        p = torch.from_numpy(np.ascontiguousarray(b.params)).cuda() if b.params.size else None
        u = torch.from_numpy(np.ascontiguousarray(b.u0)).cuda()
        st = torch.empty(b.batch, dtype=torch.int32, device="cuda")
        it = torch.empty(b.batch, dtype=torch.int32, device="cuda")
        held.append((p, u, st, it))
        reqs.append(solver.submit(b.family, p, u, alg, 1e-10, 50, (st, it, None, None)))
    solver.flush()
    solved = [solver.wait(r) for r in reqs]
    return [(u.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy(), s)
            for (p, u, st, it), s in zip(held, solved)]


@pytest.mark.parametrize("alg", [LS, LS | MIXED, TR | MIXED])
def test_mix_equals_alone(solver, alg):
    batches = I.uneven_batches(1 << 13, config_id=2)
    mixed = submit_all(solver, batches, alg)
    for b, (u, st, it, s) in zip(batches, mixed):
        alone = gpu_solve(solver, b, alg)
        np.testing.assert_array_equal(u, alone["u"])
        np.testing.assert_array_equal(st, alone["status"])
        np.testing.assert_array_equal(it, alone["iters"])
        assert s == alone["solved"]


@pytest.mark.parametrize("base", [LS, TR])
def test_fp64_and_mixed_buckets_in_one_flush(solver, base):
    # every bucket of an uneven batch twice, once in FP64 and once in mixed
    # precision, plus a per-bucket choice (mixed for the odd buckets), all in
    # one flush: each request equals the same request solved alone
    batches = I.uneven_batches(1 << 13, config_id=2)
    both = batches + batches + batches
    algs = ([base] * len(batches) + [base | MIXED] * len(batches)
            + [base | (MIXED if i % 2 else 0) for i in range(len(batches))])
    res = submit_all(solver, both, algs)
    for b, a, (u, st, it, s) in zip(both, algs, res):
        alone = gpu_solve(solver, b, a)
        np.testing.assert_array_equal(u, alone["u"])
        np.testing.assert_array_equal(st, alone["status"])
        np.testing.assert_array_equal(it, alone["iters"])
        assert s == alone["solved"] == b.batch


def test_graph_and_direct_agree(solver):
    import paper_2403_16341_gb300 as nls
    batches = I.uneven_batches(1 << 12, config_id=2)
    a = submit_all(solver, batches, TR)
    solver.set_option(nls.NLS_OPT_GRAPH, 0)
    b = submit_all(solver, batches, TR)
    solver.set_option(nls.NLS_OPT_GRAPH, 1)
    for x, y in zip(a, b):
        for i in range(3):
            np.testing.assert_array_equal(x[i], y[i])
        assert x[3] == y[3]


def test_cached_graph_reused_with_new_data(solver):
    # same shape, different instances: the cached executable graph is updated
    for seed in (0, 1, 2):
        batches = [I.cubic_batch(n, 1000, seed=seed, config_id=6) for n in (3, 8, 12)]
        res = submit_all(solver, batches, LS)
        for b, (u, st, it, s) in zip(batches, res):
            o = oracle_solve(b, LS)
            g = {"u": u, "status": st, "iters": it, "resid": np.zeros(b.batch), "solved": s}
            ok = st == 0
            np.testing.assert_array_equal(st, o["status"])
            assert np.abs(u[:, ok] - o["u"][:, ok]).max() < 1e-9


@pytest.mark.parametrize("n", [3, 8, 12, 24, 40])
def test_autotune_choice_is_valid_and_used(solver, n, tmp_path):
    import torch
    import paper_2403_16341_gb300 as nls
    b = I.cubic_batch(n, 4096, config_id=7) if n <= 32 else I.bratu_batch(n, 2048, config_id=7)
    p = torch.from_numpy(b.params).cuda()
    u = torch.from_numpy(b.u0).cuda()
    u_before = u.clone()
    tiles = solver.autotune(b.family, p, u, LS | MIXED)
    assert torch.equal(u, u_before)  # the tuner restores u
    allowed = {nls.NLS_TILE_THREAD, nls.NLS_TILE_WARP, nls.NLS_TILE_CTA}
    assert tiles in allowed
    if n > 32:
        assert tiles == nls.NLS_TILE_CTA
    if n > 8:
        assert tiles != nls.NLS_TILE_THREAD
    g = gpu_solve(solver, b, LS | MIXED)
    check_parity(b, g, oracle_solve(b, LS), mixed=True)
    path = str(tmp_path / "tune.txt")
    nls.nls_tune_save(solver.h, path)
    text = open(path).read()
    assert f" {n} " in text
    s2 = nls.Solver(0)
    nls.nls_tune_load(s2.h, path)
    g2 = gpu_solve(s2, b, LS | MIXED)
    s2.close()
    np.testing.assert_array_equal(g2["u"], g["u"])


@pytest.mark.parametrize("mixed", [False, True])
def test_uneven_full_size(solver, mixed):
    # 2^18 instances, n log-uniform in 2..32, half cubic and half Bratu,
    # NR + backtracking, all buckets in one flush
    batches = I.workload_uneven()
    assert sum(b.batch for b in batches) == 1 << 18
    alg = LS | (MIXED if mixed else 0)
    res = submit_all(solver, batches, alg)
    rng = np.random.default_rng(3)
    total = 0
    for b, (u, st, it, s) in zip(batches, res):
        assert (st == 0).all() and s == b.batch
        total += s
        idx = np.sort(rng.choice(b.batch, min(3, b.batch), replace=False))
        sub = I.Batch(b.family, b.n, b.params[:, idx], b.u0[:, idx])
        p = sub.params
        for j, k in enumerate(idx):
            F = O.residual(b.family, p[:, j] if p.size else np.zeros(1), u[:, k])
            assert np.abs(F).max() <= 1e-10
        o = oracle_solve(sub, LS)
        ref = O.polish_batch(b.family, sub.params, o["u"])
        err = np.abs(u[:, idx] - ref).max(axis=0) / np.maximum(1, np.abs(ref).max(axis=0))
        assert err.max() <= (1e-8 if mixed else 1e-9)
    assert total == 1 << 18


def test_uneven_full_size_fp64_and_mixed_in_one_flush(solver):
    # the 2^18-instance uneven set solved in FP64 and in mixed precision in
    # one flush (124 requests): every instance solved in both precisions, a
    # sample of each bucket within the parity tolerance of its precision
    batches = I.workload_uneven()
    algs = [LS] * len(batches) + [LS | MIXED] * len(batches)
    res = submit_all(solver, batches + batches, algs)
    rng = np.random.default_rng(5)
    for j, b in enumerate(batches):
        idx = np.sort(rng.choice(b.batch, min(3, b.batch), replace=False))
        sub = I.Batch(b.family, b.n, b.params[:, idx], b.u0[:, idx])
        o = oracle_solve(sub, LS)
        ref = O.polish_batch(b.family, sub.params, o["u"])
        for (u, st, it, s), tol in ((res[j], 1e-9), (res[len(batches) + j], 1e-8)):
            assert (st == 0).all() and s == b.batch
            err = np.abs(u[:, idx] - ref).max(axis=0) / np.maximum(1, np.abs(ref).max(axis=0))
            assert err.max() <= tol


@pytest.mark.parametrize("n,alg", [(6, 5), (12, 5), (40, 4), (24, 7)])
def test_autotune_next4_algorithms(solver, n, alg, tmp_path):
    # Halley, Potra-Ptak and modified Broyden: the tuner picks among the
    # tilings that hold n and the solve it then runs matches the oracle
    import torch
    import paper_2403_16341_gb300 as nls
    b = I.cubic_batch(n, 2048, config_id=7)
    p = torch.from_numpy(b.params).cuda()
    u = torch.from_numpy(b.u0).cuda()
    tiles = solver.autotune(b.family, p, u, alg | MIXED)
    assert tiles in {nls.NLS_TILE_THREAD, nls.NLS_TILE_WARP, nls.NLS_TILE_CTA}
    if n > 8:
        assert tiles != nls.NLS_TILE_THREAD
    if n > 32:
        assert tiles == nls.NLS_TILE_CTA
    g = gpu_solve(solver, b, alg | MIXED)
    check_parity(b, g, oracle_solve(b, alg), mixed=True)
    path = str(tmp_path / "tune.txt")
    nls.nls_tune_save(solver.h, path)
    s2 = nls.Solver(0)
    nls.nls_tune_load(s2.h, path)
    g2 = gpu_solve(s2, b, alg | MIXED)
    s2.close()
    np.testing.assert_array_equal(g2["u"], g["u"])

