"""The per-instance count of trust-region passes that formed the dogleg's
gradient g = J^T F and J g (nls_outputs.ngrad), against the oracle's trace.

The thread tiling forms g only when the Newton step leaves the region, once
per Jacobian; the warp and CTA tilings form it with every new Jacobian.  A
new Jacobian is taken at the first pass and after every accepted step
(Sec. 2.2.2: a rejected step only shrinks the region and reuses J)."""
import numpy as np
import pytest

import oracle as O
from paper_2403_16341_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NEWTON, LS, TR = 0, 1, 2
MIXED = 1 << 8
TILE_THREAD, TILE_WARP, TILE_CTA = 1 << 10, 1 << 11, 1 << 12


def expected_counts(b, k):
    """(passes with a new Jacobian, of those the ones whose epoch reached the
    boundary) from the oracle's trace of instance k."""
    p = b.params[:, k] if b.params.size else np.zeros(1)
    t = O.solve_trace(b.family, p, b.u0[:, k], O.ALG_TRUST_DOGLEG)
    epochs, boundary = 0, 0
    new_j, hit = True, False
    for br, rho in zip(t["branch"], t["rho"]):
        if new_j:
            epochs += 1
            hit = False
            new_j = False
        if br != 0 and not hit:
            boundary += 1
            hit = True
        if rho > 0.0:  # accepted: the next pass takes a new Jacobian
            new_j = True
    return t["status"], t["iters"], epochs, boundary


def gpu_counts(b, alg):
    import torch
    import paper_2403_16341_gb300 as nls
    s = nls.Solver(0)
    p = torch.from_numpy(np.ascontiguousarray(b.params)).cuda()
    u = torch.from_numpy(np.ascontiguousarray(b.u0)).cuda()
    outs = [torch.empty(b.batch, dtype=torch.int32, device="cuda") for _ in range(2)]
    ng = torch.full((b.batch,), -1, dtype=torch.int32, device="cuda")
    s.wait(s.submit(b.family, p, u, alg, 1e-10, 50, (outs[0], outs[1], None, None, ng)))
    s.close()
    return outs[0].cpu().numpy(), outs[1].cpu().numpy(), ng.cpu().numpy()


@pytest.mark.parametrize("n,tile,lazy", [(8, TILE_THREAD, True), (3, TILE_THREAD, True),
                                         (12, TILE_WARP, False), (40, TILE_CTA, False)])
def test_gradient_passes_match_the_trace(n, tile, lazy):
    b = I.cubic_batch(n, 300, config_id=1, b_half_width=5.0 if n == 8 else 2.0)
    st, it, ng = gpu_counts(b, TR | tile)
    same, hits = 0, 0
    for k in range(b.batch):
        ost, oit, epochs, boundary = expected_counts(b, k)
        if ost != st[k] or oit != it[k]:
            continue
        same += 1
        want = boundary if lazy else epochs
        assert ng[k] == want, (k, ng[k], want, epochs, boundary)
        hits += want > 0
    assert same > 0.95 * b.batch and hits > 0


@pytest.mark.parametrize("alg", [NEWTON, LS, TR | MIXED, 5, 3])
def test_gradient_passes_other_algorithms(alg):
    b = I.cubic_batch(8, 200, config_id=1, b_half_width=5.0)
    st, it, ng = gpu_counts(b, alg)
    if alg == TR | MIXED:
        assert (ng >= 0).all() and (ng <= it).all() and ng.sum() > 0
    else:
        # Newton, backtracking, Halley and the poly-algorithm form no dogleg gradient
        assert (ng == 0).all()
