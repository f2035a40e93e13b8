"""The FP64 pivot reciprocal (FP32 seed + two Newton-Raphson steps) stays
within one ulp of the correctly rounded 1/x over the whole exponent range,
and matches special cases exactly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_rcp_within_one_ulp():
    import torch
    import paper_2403_16341_gb300 as nls
    rng = np.random.default_rng(0)
    mant = rng.uniform(1.0, 2.0, 1 << 20)
    expo = rng.integers(-1000, 1000, 1 << 20)
    sign = rng.choice([-1.0, 1.0], 1 << 20)
    x = np.ldexp(mant, expo) * sign
    x = np.concatenate([x, [1.0, -1.0, 3.0, 0.1, 1e-300, 1e300, 2.0 ** -1022, 5e-324,
                            0.0, -0.0, np.inf, -np.inf, np.nan]])
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    nls.nls_probe_rcp(xd.data_ptr(), yd.data_ptr(), x.size)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
        ref = 1.0 / x
    finite = np.isfinite(ref) & (ref != 0)
    ulps = np.abs(y[finite] - ref[finite]) / np.spacing(np.abs(ref[finite]))
    assert ulps.max() <= 1.0, ulps.max()
    special = ~finite
    np.testing.assert_array_equal(np.isnan(y[special]), np.isnan(ref[special]))
    ok = ~np.isnan(ref[special])
    np.testing.assert_array_equal(y[special][ok], ref[special][ok])
