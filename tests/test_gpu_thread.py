"""GPU parity of the thread-tiled solver (n <= 8) against the FP64 oracle,
through the C ABI.  Tolerances: 1e-9 (FP64) and 1e-8 (mixed) relative to
max(1, ||u*||_inf); identical status sets in FP64, a superset in mixed."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2403_16341_gb300 import inputs as I
from tests.parity import check_parity, gpu_solve, oracle_solve

pytestmark = pytest.mark.gpu

NEWTON, LS, TR = 0, 1, 2
MIXED, ANALYTIC = 1 << 8, 1 << 9


@pytest.fixture(scope="module")
def solver():
    import paper_2403_16341_gb300 as nls
    s = nls.Solver(0)
    yield s
    s.close()


@pytest.mark.parametrize("jac", [0, ANALYTIC])
def test_cubic_n3_1024_newton_fp64(solver, jac):
    b = I.workload_cubic_n3()
    g = gpu_solve(solver, b, NEWTON | jac)
    o = oracle_solve(b, NEWTON)
    check_parity(b, g, o, mixed=False)
    assert g["solved"] == 1024
    # FP64 mode follows the oracle's iteration for almost every instance
    assert (g["iters"] == o["iters"]).mean() > 0.99


@pytest.mark.parametrize("alg", [NEWTON, LS, TR])
@pytest.mark.parametrize("mixed", [False, True])
def test_cubic_n8_parity(solver, alg, mixed):
    b = I.cubic_batch(8, 4099, config_id=1, b_half_width=5.0)  # ragged tail
    g = gpu_solve(solver, b, alg | (MIXED if mixed else 0))
    o = oracle_solve(b, alg)
    err = check_parity(b, g, o, mixed)
    assert g["solved"] == b.batch
    print(f"alg {alg} mixed {mixed}: max rel err {err.max():.2e}, "
          f"mean iters gpu {g['iters'].mean():.2f} oracle {o['iters'].mean():.2f}")


@pytest.mark.parametrize("family", [I.FAMILY_CUBIC, I.FAMILY_BRATU, I.FAMILY_SQUARE,
                                    I.FAMILY_ROSENBROCK])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("alg", [NEWTON, LS, TR])
@pytest.mark.parametrize("mode", [0, MIXED, ANALYTIC])
def test_families_all_sizes(solver, family, n, alg, mode):
    B = 97
    if family == I.FAMILY_CUBIC:
        b = I.cubic_batch(n, B, config_id=2)
    elif family == I.FAMILY_BRATU:
        if n == 1:
            pytest.skip("discrete Bratu with n = 1 has no root for lambda > 2.94")
        b = I.bratu_batch(n, B, config_id=2)
    elif family == I.FAMILY_SQUARE:
        b = I.square_batch(n, B)
    else:
        b = I.rosenbrock_batch(n, B)
    maxiters = 200 if family == I.FAMILY_ROSENBROCK else 50
    g = gpu_solve(solver, b, alg | mode, maxiters=maxiters)
    o = oracle_solve(b, alg, maxiters=maxiters)
    check_parity(b, g, o, mixed=bool(mode & MIXED))


def test_persistent_refill_and_static_agree_bitwise(solver):
    import paper_2403_16341_gb300 as nls
    b = I.cubic_batch(8, 5000, config_id=1, b_half_width=5.0)
    runs = []
    for persistent, refill in [(0, 0), (1, 0), (1, 16), (1, 31)]:
        solver.set_option(nls.NLS_OPT_PERSISTENT, persistent)
        solver.set_option(nls.NLS_OPT_REFILL_BELOW, refill)
        runs.append(gpu_solve(solver, b, TR | MIXED))
    solver.set_option(nls.NLS_OPT_PERSISTENT, 1)
    solver.set_option(nls.NLS_OPT_REFILL_BELOW, 24)
    for r in runs[1:]:
        for key in ("u", "status", "iters", "resid", "nfev"):
            np.testing.assert_array_equal(r[key], runs[0][key])


def test_deterministic(solver):
    b = I.cubic_batch(8, 3000, config_id=1, b_half_width=5.0)
    r1 = gpu_solve(solver, b, LS)
    r2 = gpu_solve(solver, b, LS)
    for key in ("u", "status", "iters", "resid", "nfev"):
        np.testing.assert_array_equal(r1[key], r2[key])


def test_edge_cases(solver):
    # batch 1, NaN parameter, maxiters 0, converged start, singular Jacobian
    b = I.cubic_batch(2, 1, config_id=3)
    g = gpu_solve(solver, b, NEWTON)
    assert g["status"][0] == 0
    bad = I.cubic_batch(2, 4, config_id=3)
    bad.params[5, 1] = np.nan
    g = gpu_solve(solver, bad, TR)
    assert g["status"][1] == O.ST_NONFINITE and (np.delete(g["status"], 1) == 0).all()
    g = gpu_solve(solver, b, NEWTON, maxiters=0)
    assert g["status"][0] == O.ST_MAXITERS and g["iters"][0] == 0
    root = gpu_solve(solver, b, NEWTON)["u"]
    b2 = I.Batch(b.family, b.n, b.params, root)
    g = gpu_solve(solver, b2, LS, maxiters=0)
    assert g["status"][0] == O.ST_SUCCESS and g["iters"][0] == 0
    sq = I.Batch(I.FAMILY_SQUARE, 3, np.full((3, 2), 2.0), np.zeros((3, 2)))
    g = gpu_solve(solver, sq, NEWTON)
    assert (g["status"] == O.ST_SINGULAR).all() and (g["iters"] == 1).all()
    # Rosenbrock from (-1.2, 1, ..): plain Newton overflows, backtracking converges (Fig. 1)
    u0 = np.ones((8, 1))
    u0[0] = -1.2
    rb = I.Batch(I.FAMILY_ROSENBROCK, 8, np.zeros((0, 1)), u0)
    assert gpu_solve(solver, rb, NEWTON, 1e-8, 1000)["status"][0] == O.ST_NONFINITE
    g = gpu_solve(solver, rb, LS, 1e-8, 1000)
    assert g["status"][0] == O.ST_SUCCESS and np.abs(g["u"] - 1).max() < 1e-9


def test_empty_batch(solver):
    import torch
    u = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    p = torch.zeros((12, 0), dtype=torch.float64, device="cuda")
    req = solver.submit(0, p, u, NEWTON)
    assert solver.wait(req) == 0


def test_api_errors(solver):
    import paper_2403_16341_gb300 as nls
    import torch
    u = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    p = torch.zeros((12, 4), dtype=torch.float64, device="cuda")
    cases = [
        (dict(family=9), nls.NLS_E_UNSUPPORTED), (dict(n=0), nls.NLS_E_UNSUPPORTED),
        (dict(n=129), nls.NLS_E_UNSUPPORTED), (dict(batch=-1), nls.NLS_E_INVALID),
        (dict(alg=8), nls.NLS_E_INVALID), (dict(abstol=-1.0), nls.NLS_E_INVALID),
        (dict(abstol=float("nan")), nls.NLS_E_INVALID), (dict(maxiters=-1), nls.NLS_E_INVALID),
        (dict(u=0), nls.NLS_E_INVALID), (dict(params=0), nls.NLS_E_INVALID),
    ]
    base = dict(family=0, params=p.data_ptr(), u=u.data_ptr(), n=3, batch=4, alg=0,
                abstol=1e-10, maxiters=50)
    for over, code in cases:
        kw = dict(base, **over)
        with pytest.raises(nls.NlsError) as e:
            nls.nls_solve(solver.h, kw["family"], kw["params"], kw["u"], kw["n"], kw["batch"],
                          kw["alg"], kw["abstol"], kw["maxiters"])
        assert e.value.code == code, (over, e.value)
    with pytest.raises(nls.NlsError) as e:
        nls.nls_status(solver.h, 123456789)
    assert e.value.code == nls.NLS_E_NOTFOUND


@pytest.mark.parametrize("case", ["small", "chunked", "chunked_warp"])
def test_host_entry_point_matches_device(solver, case):
    # batches of 2^18 instances and more are pipelined in chunks of at least
    # 2^17 (copies on their own streams); the results equal the device-buffer path
    import ctypes
    import paper_2403_16341_gb300 as nls
    if case == "small":
        b, alg = I.cubic_batch(8, 2000, config_id=1, b_half_width=5.0), TR | MIXED
    elif case == "chunked":
        b, alg = I.cubic_batch(8, 300001, config_id=1, b_half_width=5.0), TR | MIXED
    else:
        b, alg = I.bratu_batch(12, 270001, config_id=2), LS
    g = gpu_solve(solver, b, alg)
    u = np.ascontiguousarray(b.u0.copy())
    st = np.zeros(b.batch, dtype=np.int32)
    it = np.zeros(b.batch, dtype=np.int32)
    rs = np.zeros(b.batch)
    nf = np.zeros(b.batch, dtype=np.int32)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p).value
    solved = nls.nls_solve_host(solver.h, b.family, ptr(b.params), ptr(u), b.n, b.batch,
                                alg, 1e-10, 50, ptr(st), ptr(it), ptr(rs), ptr(nf))
    assert solved == g["solved"]
    np.testing.assert_array_equal(u, g["u"])
    np.testing.assert_array_equal(st, g["status"])
    np.testing.assert_array_equal(it, g["iters"])
    np.testing.assert_array_equal(rs, g["resid"])
    np.testing.assert_array_equal(nf, g["nfev"])


def test_host_request_full_size_eight_chunks(solver):
    # the end-to-end path of the benchmark: 2^20 instances on pinned host
    # buffers, eight chunks whose solves alternate between two streams;
    # every output equals the device-buffer path, bit for bit
    import torch
    import paper_2403_16341_gb300 as nls
    b = I.cubic_batch(8, 1 << 20, config_id=1, b_half_width=5.0)
    for alg in (TR, LS | MIXED):
        ref = gpu_solve(solver, b, alg)
        hp = torch.from_numpy(np.ascontiguousarray(b.params)).pin_memory()
        hu = torch.from_numpy(np.ascontiguousarray(b.u0)).pin_memory()
        hst = torch.zeros(b.batch, dtype=torch.int32).pin_memory()
        hit = torch.zeros(b.batch, dtype=torch.int32).pin_memory()
        req = nls.nls_solve_host_async(solver.h, b.family, hp.data_ptr(), hu.data_ptr(), b.n, b.batch, alg,
                                       1e-10, 50, hst.data_ptr(), hit.data_ptr())
        assert nls.nls_status(solver.h, req) == ref["solved"] == b.batch
        np.testing.assert_array_equal(hu.numpy(), ref["u"])
        np.testing.assert_array_equal(hst.numpy(), ref["status"])
        np.testing.assert_array_equal(hit.numpy(), ref["iters"])


def test_pending_device_request_then_chunked_host_request(solver):
    # a device-buffer request made with nls_solve and not yet flushed is
    # launched on the handle's stream before a host request's chunks, which
    # alternate between two solve streams; both equal their requests made
    # alone
    import torch
    import paper_2403_16341_gb300 as nls
    bd = I.cubic_batch(8, 70001, config_id=1, b_half_width=5.0)
    bh = I.cubic_batch(8, 300001, config_id=2, b_half_width=5.0)  # two chunks
    ref_d, ref_h = gpu_solve(solver, bd, LS | MIXED), gpu_solve(solver, bh, TR)
    dev = torch.device("cuda", 0)
    p = torch.from_numpy(np.ascontiguousarray(bd.params)).to(dev)
    u = torch.from_numpy(np.ascontiguousarray(bd.u0)).to(dev)
    st = torch.empty(bd.batch, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    rd = solver.submit(bd.family, p, u, LS | MIXED, outputs=(st, None, None, None))
    hp = torch.from_numpy(np.ascontiguousarray(bh.params)).pin_memory()
    hu = torch.from_numpy(np.ascontiguousarray(bh.u0)).pin_memory()
    hst = torch.zeros(bh.batch, dtype=torch.int32).pin_memory()
    rh = nls.nls_solve_host_async(solver.h, bh.family, hp.data_ptr(), hu.data_ptr(), bh.n, bh.batch, TR,
                                  1e-10, 50, hst.data_ptr())
    assert nls.nls_status(solver.h, rh) == ref_h["solved"]
    assert solver.wait(rd) == ref_d["solved"]
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hu.numpy(), ref_h["u"])
    np.testing.assert_array_equal(hst.numpy(), ref_h["status"])
    np.testing.assert_array_equal(u.cpu().numpy(), ref_d["u"])
    np.testing.assert_array_equal(st.cpu().numpy(), ref_d["status"])


def test_host_async_requests_pipeline(solver):
    # several host requests in flight at once (pinned buffers, chunked and
    # not, different algorithms and families): each equals the device-buffer
    # path, whatever order they are waited for in; a poll before completion
    # may time out, and a finished id is released
    import ctypes
    import torch
    import paper_2403_16341_gb300 as nls
    cases = [(I.cubic_batch(8, 300001, config_id=1, b_half_width=5.0), TR | MIXED),
             (I.cubic_batch(8, 300001, config_id=1, b_half_width=5.0), LS),
             (I.bratu_batch(12, 5001, config_id=2), LS | MIXED),
             (I.cubic_batch(3, 1024, config_id=0), NEWTON)]
    ptr = lambda t: t.data_ptr() if t.numel() else 0
    held, reqs = [], []
    for b, alg in cases:
        p = torch.from_numpy(np.ascontiguousarray(b.params)).pin_memory()
        u = torch.from_numpy(np.ascontiguousarray(b.u0)).pin_memory()
        st = torch.zeros(b.batch, dtype=torch.int32).pin_memory()
        it = torch.zeros(b.batch, dtype=torch.int32).pin_memory()
        rs = torch.zeros(b.batch, dtype=torch.float64).pin_memory()
        held.append((p, u, st, it, rs))
        reqs.append(nls.nls_solve_host_async(solver.h, b.family, ptr(p), ptr(u), b.n, b.batch, alg,
                                             1e-10, 50, ptr(st), ptr(it), ptr(rs)))
    # a poll: None while in flight; once it reports completion the id is released
    first = nls.nls_status(solver.h, reqs[0], 0)
    assert first is None or first >= 0
    polled = {0: first} if first is not None else {}
    for i in (3, 1, 0, 2):
        (b, alg), (p, u, st, it, rs) = cases[i], held[i]
        solved = polled[i] if i in polled else nls.nls_status(solver.h, reqs[i])
        g = gpu_solve(solver, b, alg)
        assert solved == g["solved"]
        np.testing.assert_array_equal(u.numpy(), g["u"])
        np.testing.assert_array_equal(st.numpy(), g["status"])
        np.testing.assert_array_equal(it.numpy(), g["iters"])
        np.testing.assert_array_equal(rs.numpy(), g["resid"])
        with pytest.raises(nls.NlsError) as e:
            nls.nls_status(solver.h, reqs[i])
        assert e.value.code == nls.NLS_E_NOTFOUND


def test_grouped_requests(solver):
    # several requests flushed together complete independently and equal solo runs
    import torch
    bs = [I.cubic_batch(n, 700 + 13 * n, config_id=5) for n in (2, 5, 8)]
    solo = [gpu_solve(solver, b, LS | MIXED) for b in bs]
    us, reqs = [], []
    for b in bs:
        p = torch.from_numpy(b.params).cuda()
        u = torch.from_numpy(b.u0).cuda()
        us.append((p, u))
        reqs.append(solver.submit(b.family, p, u, LS | MIXED))
    solver.flush()
    for (p, u), req, s in zip(us, reqs, solo):
        assert solver.wait(req) == s["solved"]
        np.testing.assert_array_equal(u.cpu().numpy(), s["u"])


@pytest.mark.parametrize("alg", [LS, TR])
@pytest.mark.parametrize("mixed", [False, True])
def test_cubic_n8_full_size_sampled(solver, alg, mixed):
    # the 2^20-instance workload in the benchmark's launch configuration;
    # the oracle solves a sample of instances one by one
    b = _full_cubic_n8()
    g = gpu_solve(solver, b, alg | (MIXED if mixed else 0))
    assert g["solved"] == b.batch
    assert (g["resid"] <= 1e-10).all()
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(b.batch, 3000, replace=False))
    sub = I.Batch(b.family, b.n, b.params[:, idx], b.u0[:, idx])
    gs = {k: (v[:, idx] if k == "u" else v[idx]) for k, v in g.items() if k != "solved"}
    gs["solved"] = int((gs["status"] == 0).sum())
    o = oracle_solve(sub, alg)
    check_parity(sub, gs, o, mixed)


@functools.lru_cache(maxsize=1)
def _full_cubic_n8():
    return I.workload_cubic_n8()
