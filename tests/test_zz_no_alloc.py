"""rqb_sketch_noalloc: the sketch step for callers that cannot allocate device
memory (the allocator is off limits to them, or owned and capped by someone
else).  It keeps its scratch in one static device array instead of asking for
memory, so it must give the same Y and ||A||_F^2 as rqb_sketch and as the oracle's
sketch, call after call, even though every call reuses (and leaves behind) the
same scratch.

This file is collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from parity_util import assert_elementwise, product_bound, to_dev, to_np

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-5), (torch.float64, 1e-12)])
def test_noalloc_matches_rqb_sketch_two_calls(orc, rqb_lib, dtype, tol):
    rng = np.random.default_rng(17)
    f32 = dtype == torch.float32
    prec = 32 if f32 else 64
    # several shapes in a row, so that each call runs on the scratch the
    # previous one left behind: 128-row tiles with split-K partials (3001 rows
    # give 24 row tiles, fewer than the SMs), 37 ragged columns, and for FP32
    # the 64-row tiles of a 256-column product; one call without the norm
    cases = [(3001, 2049, 0, 128 if f32 else 64, 7, True),
             (517, 1800, 64, 37, 8, True),
             (700, 900, 5, 256 if f32 else 128, 9, False),
             (3001, 2049, 0, 128 if f32 else 64, 7, True)]
    with rqb_lib.Handle(dtype) as h:
        for (m, n, col0, p, seed, want_norm) in cases:
            A = rng.standard_normal((m, n))
            if f32:
                A = A.astype(np.float32).astype(np.float64)
            Ad = to_dev(A, dtype)
            Yref, nref = h.rqb_sketch(Ad, col0, p, seed)
            Y = rqb_lib.colmajor(torch.full((p, m), float("nan"), dtype=dtype, device="cuda").t())
            rc, nrm = rqb_lib.rqb_sketch_noalloc(Ad, col0, p, seed, Y, want_norm=want_norm)
            torch.cuda.synchronize()
            assert rc == rqb_lib.RQB_OK, rqb_lib.status_string(rc)
            Yg = to_np(Y)
            # the oracle's sketch on the same Omega (up to the generators'
            # last-ulp differences), entry by entry
            Yo = orc.sketch(A, seed, col0, p, omega_prec=prec)
            Om = orc.omega(seed, n, col0, p, prec=prec)
            if f32:
                dOm = 4 * np.spacing(np.abs(Om).astype(np.float32)).astype(np.float64) + 1e-7
            else:
                dOm = 5e-14 * max(1.0, np.abs(Om).max()) * np.ones_like(Om)
            assert_elementwise(Yg, Yo, product_bound(A, Om), 1e-6 if f32 else 1e-14, "no-alloc sketch",
                               extra=np.abs(A) @ dOm)
            # and the handle's sketch step
            assert _rel(Yg, to_np(Yref)) <= tol
            if want_norm:
                assert abs(nrm - nref) <= tol * nref
                assert abs(nrm - np.sum(A * A)) <= (1e-9 if f32 else 1e-12) * np.sum(A * A)
            else:
                assert nrm is None


def test_noalloc_rejects_sizes_beyond_scratch(rqb_lib):
    A = torch.zeros(64, 1, dtype=torch.float32, device="cuda")
    Y = torch.zeros(64, 128, dtype=torch.float32, device="cuda").t().contiguous().t()
    import ctypes
    # n * 128 floats of Omega alone exceed the fixed scratch: rejected before any launch
    n_huge = 1 << 20
    rc = rqb_lib.lib().rqb_sketch_noalloc(rqb_lib.RQB_F32, ctypes.c_void_p(A.data_ptr()), 64, n_huge, 64, 0, 128, 0,
                                          ctypes.c_void_p(Y.data_ptr()), 64, None, None)
    assert rc == rqb_lib.RQB_ERR_SCRATCH_LIMIT
    rc = rqb_lib.lib().rqb_sketch_noalloc(rqb_lib.RQB_F32, ctypes.c_void_p(A.data_ptr()), 64, 1, 63, 0, 8, 0,
                                          ctypes.c_void_p(Y.data_ptr()), 64, None, None)
    assert rc == rqb_lib.RQB_ERR_INVALID
