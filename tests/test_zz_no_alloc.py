"""The allocation-free entry point nls_solve_noalloc, called through the C
ABI, gives the same results as nls_solve on the same inputs, on two calls
in a row (the second call reuses the static scratch the first one left).

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone."""
import numpy as np
import pytest

from paper_2403_16341_gb300 import inputs as I
from tests.parity import FP64_TOL, MIXED_TOL, gpu_solve, rel_err

pytestmark = pytest.mark.gpu

NEWTON, LS, TR = 0, 1, 2
MIXED = 1 << 8


def _device_group(torch, b):
    p = torch.from_numpy(np.ascontiguousarray(b.params)).cuda()
    u = torch.from_numpy(np.ascontiguousarray(b.u0)).cuda()
    outs = (torch.empty(b.batch, dtype=torch.int32, device="cuda"),
            torch.empty(b.batch, dtype=torch.int32, device="cuda"),
            torch.empty(b.batch, dtype=torch.float64, device="cuda"),
            torch.empty(b.batch, dtype=torch.int32, device="cuda"))
    return p, u, outs


@pytest.mark.parametrize("alg", [NEWTON | MIXED, TR, TR | MIXED, LS, TR | (1 << 13)])
def test_noalloc_matches_handle_path_twice(alg):
    import torch
    import paper_2403_16341_gb300 as nls

    batches = [I.cubic_batch(8, 3001, config_id=1, b_half_width=5.0),
               I.cubic_batch(3, 1024, config_id=0),
               I.bratu_batch(6, 517, config_id=2)]
    solver = nls.Solver(0)
    ref = [gpu_solve(solver, b, alg) for b in batches]
    solver.close()
    stream = torch.cuda.current_stream().cuda_stream
    tol = MIXED_TOL if alg & MIXED else FP64_TOL
    for call in range(2):
        dev = [_device_group(torch, b) for b in batches]
        groups = [(b.family, b.n, p.data_ptr(), u.data_ptr(), b.batch,
                   tuple(t.data_ptr() for t in outs)) for b, (p, u, outs) in zip(batches, dev)]
        solved = nls.nls_solve_noalloc(stream, groups, alg, 1e-10, 50)
        torch.cuda.synchronize()
        for b, r, s, (p, u, outs) in zip(batches, ref, solved, dev):
            st, it, rs, nf = (t.cpu().numpy() for t in outs)
            assert s == r["solved"] == b.batch, (call, s, r["solved"])
            np.testing.assert_array_equal(st, r["status"])
            np.testing.assert_array_equal(it, r["iters"])
            np.testing.assert_array_equal(nf, r["nfev"])
            assert rel_err(u.cpu().numpy(), r["u"]).max() <= tol
            assert (rs <= 1e-10).all()


def test_noalloc_rejects_too_many_groups():
    import torch
    import paper_2403_16341_gb300 as nls
    u = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    p = torch.zeros((12, 4), dtype=torch.float64, device="cuda")
    g = (0, 3, p.data_ptr(), u.data_ptr(), 4, (0, 0, 0, 0))
    with pytest.raises(nls.NlsError) as e:
        nls.nls_solve_noalloc(0, [g] * (nls.NLS_NOALLOC_MAX_GROUPS + 1), NEWTON, 1e-10, 50)
    assert e.value.code == nls.NLS_E_INVALID and "groups" in str(e.value)
    big = (0, 9, p.data_ptr(), u.data_ptr(), 4, (0, 0, 0, 0))
    with pytest.raises(nls.NlsError) as e:
        nls.nls_solve_noalloc(0, [big], NEWTON, 1e-10, 50)
    assert e.value.code == nls.NLS_E_UNSUPPORTED
    # the other algorithms of nls_solve are not run here; unknown ones are invalid
    for a in (nls.NLS_POLYALG, nls.NLS_POTRA_PTAK, nls.NLS_HALLEY, nls.NLS_BROYDEN,
              nls.NLS_MOD_BROYDEN):
        with pytest.raises(nls.NlsError) as e:
            nls.nls_solve_noalloc(0, [g], a, 1e-10, 50)
        assert e.value.code == nls.NLS_E_UNSUPPORTED and "only" in str(e.value)
    with pytest.raises(nls.NlsError) as e:
        nls.nls_solve_noalloc(0, [g], nls.NLS_MOD_BROYDEN + 1, 1e-10, 50)
    assert e.value.code == nls.NLS_E_INVALID
    # A = 0, b = 0: u0 = 0 is already a root of every instance
    assert nls.nls_solve_noalloc(0, [g], NEWTON, 1e-10, 50) == [4]
