"""Failure detection without a fault: a per-launch deadline stops iterating
and reports NLS_ABORTED for unfinished instances; the context stays usable."""
import numpy as np
import pytest

from paper_2403_16341_gb300 import inputs as I
from tests.parity import gpu_solve

pytestmark = pytest.mark.gpu
TR = 2
ABORTED = 6


@pytest.mark.parametrize("make,alg", [
    (lambda: I.cubic_batch(8, 1 << 18, config_id=1, b_half_width=5.0), TR),         # thread
    (lambda: I.cubic_batch(16, 1 << 14, config_id=1), TR),                          # warp
    (lambda: I.bratu_batch(96, 2048, config_id=4), TR),                             # CTA
])
def test_deadline_aborts_then_recovers(make, alg):
    import paper_2403_16341_gb300 as nls
    b = make()
    s = nls.Solver(0)
    try:
        s.set_option(nls.NLS_OPT_DEADLINE_US, 20)
        g = gpu_solve(s, b, alg)
        st = g["status"]
        assert set(np.unique(st)) <= {0, ABORTED}
        assert (st == ABORTED).any()
        assert g["solved"] == int((st == 0).sum())
        assert (g["resid"][st == 0] <= 1e-10).all()
        s.set_option(nls.NLS_OPT_DEADLINE_US, 0)
        g2 = gpu_solve(s, b, alg)
        assert (g2["status"] == 0).all()
        ok = st == 0  # instances that finished before the deadline are unchanged
        np.testing.assert_array_equal(g["u"][:, ok], g2["u"][:, ok])
    finally:
        s.close()
