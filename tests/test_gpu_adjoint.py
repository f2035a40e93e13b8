"""Adjoint sensitivity of the roots (Sec. 2.3) on the GPU, through the C ABI,
against the FP64 oracle's adjoint and the paper's example."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2403_16341_gb300 import inputs as I
from tests.parity import gpu_solve

pytestmark = pytest.mark.gpu


def gpu_adjoint(solver, family, params, u, w):
    import torch
    import paper_2403_16341_gb300 as nls
    n, B = u.shape
    E = I.n_params(family, n)
    pd = torch.from_numpy(np.ascontiguousarray(params)).cuda() if E else None
    ud = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    wd = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    gd = torch.zeros((max(E, 1), B), dtype=torch.float64, device="cuda")
    sd = torch.empty(B, dtype=torch.int32, device="cuda")
    nls.nls_adjoint(solver.h, family, pd.data_ptr() if E else 0, ud.data_ptr(), n, B,
                    wd.data_ptr(), gd.data_ptr(), sd.data_ptr())
    torch.cuda.synchronize()
    return gd.cpu().numpy()[:E], sd.cpu().numpy()


@pytest.fixture(scope="module")
def solver():
    import paper_2403_16341_gb300 as nls
    s = nls.Solver(0)
    yield s
    s.close()


def test_paper_example_gradient_is_one(solver):
    with open(os.path.join(os.path.dirname(__file__), "golden", "square_sec2_3.json")) as f:
        g = json.load(f)
    b = I.Batch(I.FAMILY_SQUARE, 2, np.array(g["p"])[:, None], np.array(g["u0"])[:, None])
    r = gpu_solve(solver, b, 0, abstol=1e-14)
    grad, st = gpu_adjoint(solver, I.FAMILY_SQUARE, b.params, r["u"], 2.0 * r["u"])
    assert st[0] == 0
    np.testing.assert_allclose(grad[:, 0], g["dg_dtheta"], rtol=1e-14)


@pytest.mark.parametrize("family", [I.FAMILY_CUBIC, I.FAMILY_BRATU, I.FAMILY_SQUARE])
@pytest.mark.parametrize("n", [1, 3, 5, 8, 9, 13, 16, 17, 32, 33, 64, 65, 100, 128])
def test_adjoint_matches_oracle(solver, family, n):
    # n <= 8: one instance per thread; n <= 32: per warp segment; n <= 128: per CTA
    if family == I.FAMILY_BRATU and n == 1:
        pytest.skip("discrete Bratu with n = 1 has no root for lambda > 2.94")
    B = 333 if n <= 32 else 97
    b = (I.cubic_batch(n, B, config_id=9) if family == I.FAMILY_CUBIC else
         I.bratu_batch(n, B, config_id=9) if family == I.FAMILY_BRATU else I.square_batch(n, B))
    # the residual scales like (n+1)^2 for Bratu: a looser stop for larger n
    r = gpu_solve(solver, b, 0, abstol=1e-13 if n <= 16 else 1e-10)
    assert (r["status"] == 0).all()
    w = np.random.default_rng(n).normal(size=(n, B))
    grad, st = gpu_adjoint(solver, family, b.params, r["u"], w)
    assert (st == 0).all()
    for k in range(B):
        ref, sing = O.adjoint(family, b.params[:, k], r["u"][:, k], w[:, k])
        assert not sing
        scale = max(1.0, np.abs(ref).max())
        # two FP64 LU solves of J^T mu = w differ by about n eps cond(J)
        # relative to mu (Bratu's J at n = 128 has cond ~ 1e4)
        J = O.jacobian(family, b.params[:, k], r["u"][:, k])
        tol = max(1e-12, 8 * n * np.finfo(float).eps * np.linalg.cond(J))
        assert np.abs(grad[:, k] - ref).max() <= tol * scale, (k, np.abs(grad[:, k] - ref).max() / scale, tol)


@pytest.mark.parametrize("n", [12, 40])
def test_adjoint_tiles_rosenbrock_status(solver, n):
    # no parameters: only the status is written; J at the root is nonsingular
    b = I.Batch(I.FAMILY_ROSENBROCK, n, np.zeros((0, 50)), np.ones((n, 50)))
    grad, st = gpu_adjoint(solver, I.FAMILY_ROSENBROCK, b.params, np.ones((n, 50)),
                           np.ones((n, 50)))
    assert (st == 0).all()


def test_adjoint_singular_and_errors(solver):
    import paper_2403_16341_gb300 as nls
    for n in (3, 12, 40):
        # square family at u = 0: J = diag(2u) = 0 on every tiling
        u = np.zeros((n, 4))
        grad, st = gpu_adjoint(solver, I.FAMILY_SQUARE, np.ones((n, 4)), u, np.ones((n, 4)))
        assert (st == O.ST_SINGULAR).all()
    # n = 129 is refused on the host, before any launch
    with pytest.raises(nls.NlsError) as e:
        nls.nls_adjoint(solver.h, 0, 1, 1, 129, 4, 1, 1)
    assert e.value.code == nls.NLS_E_UNSUPPORTED
