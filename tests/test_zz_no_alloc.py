"""rqb_sketch_noalloc: the sketch step for callers that cannot allocate device
memory (the allocator is off limits to them, or owned and capped by someone
else).  It keeps its scratch in one static device array instead of asking for
memory, so it must give the same Y and ||A||_F^2 as rqb_sketch, call after call,
even though every call reuses (and leaves behind) the same scratch.

This file is collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from parity_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-5), (torch.float64, 1e-12)])
def test_noalloc_matches_rqb_sketch_two_calls(rqb_lib, dtype, tol):
    rng = np.random.default_rng(17)
    # two different shapes in a row: the second call must not see the first's leftovers
    cases = [(3001, 2049, 0, 128 if dtype == torch.float32 else 64, 7),
             (517, 1800, 64, 37, 8)]
    with rqb_lib.Handle(dtype) as h:
        for (m, n, col0, p, seed) in cases:
            A = rng.standard_normal((m, n))
            Ad = to_dev(A, dtype)
            Yref, nref = h.rqb_sketch(Ad, col0, p, seed)
            Y = rqb_lib.colmajor(torch.full((p, m), float("nan"), dtype=dtype, device="cuda").t())
            rc, nrm = rqb_lib.rqb_sketch_noalloc(Ad, col0, p, seed, Y)
            torch.cuda.synchronize()
            assert rc == rqb_lib.RQB_OK, rqb_lib.status_string(rc)
            assert _rel(to_np(Y), to_np(Yref)) <= tol
            assert abs(nrm - nref) <= tol * nref


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
