"""The Cholesky pivots' FP64 reciprocal and reciprocal square root (an FP32
estimate refined by two Newton steps, y <- y + y (1 - d y) and
y <- y (3 - d y^2) / 2) against the correctly rounded 1/x and 1/sqrt(x) of
numpy: each step squares the relative error (2^-22 -> 2^-44 -> below the
FP64 rounding), so the results are within 2 ulp.  Inputs: random values over
the whole exponent range of the fast path (2^-120 .. 2^120), the powers of two
and their neighbours, significands near 1 and 2, and values outside that range
that take the library route."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(2026)
    parts = [np.exp2(rng.uniform(-120.0, 120.0, 200000)),
             rng.uniform(0.5, 2.0, 50000),
             np.exp2(np.arange(-130, 131, dtype=np.float64))]
    p2 = np.exp2(np.arange(-119, 120, dtype=np.float64))
    parts += [np.nextafter(p2, 0.0), np.nextafter(p2, np.inf), p2 * (1 + 2.0 ** -52), p2 * (2 - 2.0 ** -52)]
    parts += [np.array([1e-300, 1e-200, 2.0 ** -1000, 1e200, 1e300, 2.0 ** 1000, 2.0 ** -1023])]
    x = np.concatenate(parts)
    return x[x > 0]


def test_fp64_reciprocal_and_rsqrt_within_two_ulp(rqb_lib):
    x = _inputs()
    rcp, rsq = rqb_lib.rqb_fp64_recip_selftest(torch.as_tensor(x, device="cuda"))
    rcp, rsq = rcp.cpu().numpy(), rsq.cpu().numpy()
    ref_r = 1.0 / x
    ref_s = 1.0 / np.sqrt(x)
    ulp_r = np.abs(rcp - ref_r) / np.spacing(ref_r)
    ulp_s = np.abs(rsq - ref_s) / np.spacing(ref_s)
    print("max ulp: 1/x", ulp_r.max(), " 1/sqrt(x)", ulp_s.max())
    assert np.all(np.isfinite(rcp)) and np.all(np.isfinite(rsq))
    assert ulp_r.max() <= 2.0
    assert ulp_s.max() <= 2.0
