"""Parity of rqb_factor (Fig. randQB_b end to end) against the oracle.

Bars (the same seeded A and the same Omega on both sides):
  rank k              exact, unless the oracle's stopping quantity lies within
                      the GPU's decision band of eps^2 (then one block away is
                      valid, and the residual is compared with the oracle's
                      rerun at the GPU's rank in fixed-rank mode)
  residual r = ||A - QB||_F, both sides evaluated in FP64 from their own Q, B:
                      FP64 |r_gpu - r_orc| <= 1e-10 r_orc
                      FP32 |r_gpu - r_orc| <= 1e-5 ||A||_F
  ||Q^T Q - I||_max   FP64 <= 1e-12, FP32 <= 1e-5
  Q, B elementwise    FP64 (diag(R) > 0 makes Q unique): 1e-9, 1e-9 ||A||_F
Edge cases: ragged sizes (b not dividing anything, m and n off the tiles),
wide matrices, tiny matrices, padded leading dimension, rank caps
(RQB_NOT_CONVERGED), fixed-rank mode, eps = 0, invalid arguments,
rank-deficient panels (RQB_ERR_BREAKDOWN), non-finite input.
"""
import numpy as np
import pytest
import torch

import inputs
from parity_util import check_rank, oracle_at_rank, orth_err, resid, to_dev, to_np

pytestmark = pytest.mark.gpu


def _factor(rqb, A, eps, b, dtype, seed=0, lda=None, **cfg):
    with rqb.Handle(dtype, **cfg) as h:
        Q, B, k, rc = h.rqb_factor(to_dev(A, dtype, lda=lda), eps, b, seed, check=False)
        st = h.rqb_get_stats()
        return to_np(Q), to_np(B), k, rc, st


def test_fp64_config(orc, rqb_lib):
    """2000 x 1000, s_j = 10^(-8(j-1)/999), b = 50, eps = 1e-4 ||A||_F, Omega seed 0."""
    A, meta = inputs.config_fp64()
    eps, b = meta["eps"], meta["b"]
    ro = orc.randqb_b(A, eps, b, seed=0)
    Q, B, k, rc, st = _factor(rqb_lib, A, eps, b, torch.float64)
    assert rc == rqb_lib.RQB_OK
    assert k == ro.k == 600
    r_g, r_o = resid(A, Q, B), resid(A, ro.Q, ro.B)
    assert abs(r_g - r_o) <= 1e-10 * r_o
    assert r_g <= eps
    assert orth_err(Q) <= 1e-12
    assert np.abs(Q - ro.Q).max() <= 1e-9
    assert np.abs(B - ro.B).max() <= 1e-9 * np.sqrt(ro.normA2)
    assert st.blocks == ro.blocks
    assert abs(st.normA2 - ro.normA2) <= 1e-13 * ro.normA2
    np.testing.assert_allclose(st.E, ro.E, rtol=0, atol=1e-13 * ro.normA2)


@pytest.mark.parametrize("m,n,b,eps_rel", [(4000, 3200, 128, 1e-2), (4000, 3200, 128, 2e-3), (1037, 777, 37, 3e-3),
                                           (3000, 2000, 256, 1e-3), (4000, 3200, 128, 7e-4)])
def test_fp32_poly_decay(orc, rqb_lib, m, n, b, eps_rel):
    """Polynomial decay s_j = j^-1.5 (the FP32 workload's spectrum) at oracle-size;
    eps = 7e-4 ||A||_F is the multi-block benchmark point (about 12 blocks here);
    b = 256 runs the blocked Cholesky tiles (FP64 first pass, FP32 second) and
    the FP32 R^-1 from their FP32 copies."""
    s = inputs.spectrum_poly(min(m, n))
    A = inputs.usv(m, n, s, seed=m + n).astype(np.float32).astype(np.float64)
    nA = np.linalg.norm(A)
    eps = eps_rel * nA
    ro = orc.randqb_b(A, eps, b, seed=0, omega_prec=32)
    Q, B, k, rc, st = _factor(rqb_lib, A, eps, b, torch.float32)
    assert rc == rqb_lib.RQB_OK
    check_rank(k, ro, eps, b, rel_band=1e-3)
    rk = oracle_at_rank(orc, A, ro, k, b, 0, omega_prec=32)
    assert abs(resid(A, Q, B) - resid(A, rk.Q, rk.B)) <= 1e-5 * nA
    assert resid(A, Q, B) <= eps * (1 + 1e-4)
    assert orth_err(Q) <= 1e-5


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,b", [(1037, 777, 37), (500, 1500, 64), (5, 3, 2), (97, 64, 8), (300, 300, 128)])
def test_ragged_and_wide(orc, rqb_lib, dtype, m, n, b):
    r = min(m, n)
    A = inputs.usv(m, n, 0.93 ** np.arange(r), seed=m * 7 + n)
    if dtype == torch.float32:
        A = A.astype(np.float32).astype(np.float64)
    nA = np.linalg.norm(A)
    eps = 1e-2 * nA
    prec = 64 if dtype == torch.float64 else 32
    ro = orc.randqb_b(A, eps, b, seed=5, omega_prec=prec)
    Q, B, k, rc, st = _factor(rqb_lib, A, eps, b, dtype, seed=5)
    assert rc in (rqb_lib.RQB_OK, rqb_lib.RQB_NOT_CONVERGED)
    check_rank(k, ro, eps, b, rel_band=1e-6 if dtype == torch.float64 else 1e-3)
    ro = oracle_at_rank(orc, A, ro, k, b, 5, omega_prec=prec)
    if dtype == torch.float64:
        assert abs(resid(A, Q, B) - resid(A, ro.Q, ro.B)) <= 1e-10 * max(resid(A, ro.Q, ro.B), 1e-300) + 1e-14 * nA
        assert orth_err(Q) <= 1e-12
    else:
        assert abs(resid(A, Q, B) - resid(A, ro.Q, ro.B)) <= 1e-5 * nA
        assert orth_err(Q) <= 1e-5


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_padded_leading_dimension(orc, rqb_lib, dtype):
    A = inputs.usv(301, 257, 0.9 ** np.arange(257), seed=4)
    if dtype == torch.float32:
        A = A.astype(np.float32).astype(np.float64)
    eps = 1e-3 * np.linalg.norm(A)
    Q1, B1, k1, _, _ = _factor(rqb_lib, A, eps, 16, dtype, lda=333)
    Q2, B2, k2, _, _ = _factor(rqb_lib, A, eps, 16, dtype)
    assert k1 == k2
    assert np.abs(Q1 - Q2).max() <= (1e-12 if dtype == torch.float64 else 1e-5)


def test_rank_cap_not_converged(orc, rqb_lib):
    A = inputs.usv(400, 300, 0.97 ** np.arange(300), seed=8)
    Q, B, k, rc, st = _factor(rqb_lib, A, 1e-9, 16, torch.float64, max_rank=40)
    ro = orc.randqb_b(A, 1e-9, 16, seed=0, max_rank=40)
    assert rc == rqb_lib.RQB_NOT_CONVERGED and ro.status == 1
    assert k == ro.k == 40 and st.blocks == 3      # 16 + 16 + 8
    assert np.abs(Q - ro.Q).max() <= 1e-9


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_fixed_rank(orc, rqb_lib, dtype):
    A = inputs.usv(600, 400, 0.95 ** np.arange(400), seed=9)
    if dtype == torch.float32:
        A = A.astype(np.float32).astype(np.float64)
    Q, B, k, rc, st = _factor(rqb_lib, A, 1e9, 32, dtype, max_rank=100, fixed_rank=True)
    prec = 64 if dtype == torch.float64 else 32
    ro = orc.randqb_b(A, 1e9, 32, seed=0, max_rank=100, fixed_rank=True, omega_prec=prec)
    assert rc == rqb_lib.RQB_OK and k == 100 == ro.k
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    assert abs(resid(A, Q, B) - resid(A, ro.Q, ro.B)) <= tol * np.linalg.norm(A)


def test_eps_zero_runs_to_full_rank(orc, rqb_lib):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((120, 90))
    Q, B, k, rc, st = _factor(rqb_lib, A, 0.0, 32, torch.float64)
    assert k == 90 and st.blocks == 3
    assert rc in (rqb_lib.RQB_OK, rqb_lib.RQB_NOT_CONVERGED)
    assert resid(A, Q, B) <= 1e-12 * np.linalg.norm(A)
    assert orth_err(Q) <= 1e-12


def test_exact_rank_panel_breakdown(rqb_lib):
    """A panel whose Gram matrix is singular (rank(A) = 7 < b = 10) reports
    RQB_ERR_BREAKDOWN instead of producing a non-orthonormal Q."""
    A = inputs.usv(120, 90, np.arange(7, 0, -1).astype(float), seed=41)
    _, _, k, rc, _ = _factor(rqb_lib, A, 1e-12, 10, torch.float64)
    assert rc == rqb_lib.RQB_ERR_BREAKDOWN


def test_exact_rank_panel_breakdown_blocked(rqb_lib):
    """The same for a 128-wide panel, whose Gram is factored by the blocked
    multi-CTA Cholesky (rank(A) = 100 < b = 128): the failed pivot is
    reported although the elimination does not stop at it."""
    A = inputs.usv(300, 260, np.linspace(2.0, 1.0, 100), seed=43)
    _, _, k, rc, _ = _factor(rqb_lib, A, 1e-12, 128, torch.float64)
    assert rc == rqb_lib.RQB_ERR_BREAKDOWN


def test_nonfinite_input(rqb_lib):
    A = np.ones((64, 48))
    A[3, 5] = np.nan
    _, _, _, rc, _ = _factor(rqb_lib, A, 1e-3, 8, torch.float64)
    assert rc == rqb_lib.RQB_ERR_NONFINITE


def test_invalid_arguments(rqb_lib):
    import ctypes
    L = rqb_lib.lib()
    with rqb_lib.Handle(torch.float64) as h:
        A = torch.zeros(10, 8, dtype=torch.float64, device="cuda").t().contiguous().t()
        Qp, Bp = ctypes.c_void_p(), ctypes.c_void_p()
        l1, l2, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        args = lambda m, n, lda, eps, b: L.rqb_factor(h._h, ctypes.c_void_p(A.data_ptr()), m, n, lda, eps, b, 0,
                                                      ctypes.byref(Qp), ctypes.byref(l1), ctypes.byref(Bp),
                                                      ctypes.byref(l2), ctypes.byref(k))
        assert args(10, 8, 9, 1.0, 2) == rqb_lib.RQB_ERR_INVALID      # lda < m
        assert args(0, 8, 10, 1.0, 2) == rqb_lib.RQB_ERR_INVALID      # m = 0
        assert args(10, 8, 10, -1.0, 2) == rqb_lib.RQB_ERR_INVALID    # eps < 0
        assert args(10, 8, 10, 1.0, 0) == rqb_lib.RQB_ERR_INVALID     # b = 0
        assert args(10, 8, 10, 1.0, 129) == rqb_lib.RQB_ERR_INVALID   # b > 128 (FP64)
        assert args(10, 8, 10, float("nan"), 2) == rqb_lib.RQB_ERR_INVALID
        assert h.rqb_get_stats().status == rqb_lib.RQB_ERR_INVALID


def test_repeatable_bitwise(rqb_lib):
    """Deterministic reductions: two runs give identical bits."""
    A = inputs.usv(900, 700, 0.9 ** np.arange(700), seed=12).astype(np.float32).astype(np.float64)
    eps = 1e-3 * np.linalg.norm(A)
    Q1, B1, k1, _, _ = _factor(rqb_lib, A, eps, 32, torch.float32)
    Q2, B2, k2, _, _ = _factor(rqb_lib, A, eps, 32, torch.float32)
    assert k1 == k2 and np.array_equal(Q1, Q2) and np.array_equal(B1, B2)


def test_host_entry_point(orc, rqb_lib):
    A, meta = inputs.config_fp64()
    eps, b = meta["eps"], meta["b"]
    with rqb_lib.Handle(torch.float64) as h:
        Ah = torch.as_tensor(A).t().contiguous().t().pin_memory()
        cap = min(A.shape)
        Qh = torch.zeros(cap, A.shape[0], dtype=torch.float64).t()
        Bh = torch.zeros(A.shape[1], cap, dtype=torch.float64).t()
        k, rc = h.rqb_factor_host(Ah, eps, b, 0, Qh, Bh)
    ro = orc.randqb_b(A, eps, b, seed=0)
    assert rc == rqb_lib.RQB_OK and k == ro.k
    Q, B = Qh[:, :k].numpy(), Bh[:k, :].numpy()
    assert abs(resid(A, Q, B) - resid(A, ro.Q, ro.B)) <= 1e-10 * resid(A, ro.Q, ro.B)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("P", [1, 2])
def test_power_scheme_fixed_rank(orc, rqb_lib, dtype, P):
    """randQB_pb (Fig. randQB_pb) at fixed rank on the Matrix 2 spectrum (slow decay)."""
    m, n, b, k = 700, 500, 32, 96
    s = (1.0 + 200.0 * np.arange(n)) ** -0.5
    A = inputs.usv(m, n, s, seed=77)
    if dtype == torch.float32:
        A = A.astype(np.float32).astype(np.float64)
    prec = 64 if dtype == torch.float64 else 32
    ro = orc.randqb_b(A, 0.0, b, seed=3, max_rank=k, fixed_rank=True, power=P, omega_prec=prec)
    Q, B, kk, rc, st = _factor(rqb_lib, A, 0.0, b, dtype, seed=3, max_rank=k, fixed_rank=True, power=P)
    assert rc == rqb_lib.RQB_OK and kk == k == ro.k
    nA = np.linalg.norm(A)
    if dtype == torch.float64:
        assert abs(resid(A, Q, B) - resid(A, ro.Q, ro.B)) <= 1e-10 * resid(A, ro.Q, ro.B)
        assert orth_err(Q) <= 1e-12
        assert np.abs(Q - ro.Q).max() <= 1e-8
    else:
        assert abs(resid(A, Q, B) - resid(A, ro.Q, ro.B)) <= 1e-5 * nA
        assert orth_err(Q) <= 1e-5
    # the power scheme beats P = 0 at the same rank (Sec. 5.1)
    r0 = orc.randqb_b(A, 0.0, b, seed=3, max_rank=k, fixed_rank=True, power=0, omega_prec=prec)
    assert resid(A, Q, B) < resid(A, r0.Q, r0.B)


def test_power_scheme_adaptive(orc, rqb_lib):
    m, n, b = 900, 600, 40
    s = inputs.spectrum_poly(n)
    A = inputs.usv(m, n, s, seed=78)
    eps = 5e-3 * np.linalg.norm(A)
    ro = orc.randqb_b(A, eps, b, seed=1, power=1)
    Q, B, k, rc, st = _factor(rqb_lib, A, eps, b, torch.float64, seed=1, power=1)
    assert rc == rqb_lib.RQB_OK
    check_rank(k, ro, eps, b, rel_band=1e-6)
    ro = oracle_at_rank(orc, A, ro, k, b, 1, power=1)
    assert abs(resid(A, Q, B) - resid(A, ro.Q, ro.B)) <= 1e-10 * resid(A, ro.Q, ro.B)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("P", [1, 2])
def test_power_scheme_without_inner_orth(orc, rqb_lib, dtype, P):
    """Sec. 5.4 variant (RQB_FLAG_SKIP_INNER_ORTH): Y = (A A^T)^P A Omega_i and one
    orth per block.  Slow decay s_j = (1 + j)^(-1/2), so the panel's condition
    number, which grows as (sigma_1 / sigma_b)^(2P+1) within a block, stays inside
    CholeskyQR2's range; compared with the oracle's variant on the same Omega."""
    m, n, b, k = 700, 500, 32, 128
    s = (1.0 + np.arange(n)) ** -0.5
    A = inputs.usv(m, n, s, seed=79)
    if dtype == torch.float32:
        A = A.astype(np.float32).astype(np.float64)
    prec = 64 if dtype == torch.float64 else 32
    ro = orc.randqb_b(A, 0.0, b, seed=3, max_rank=k, fixed_rank=True, power=P, skip_inner_orth=True,
                      omega_prec=prec)
    Q, B, kk, rc, st = _factor(rqb_lib, A, 0.0, b, dtype, seed=3, max_rank=k, fixed_rank=True, power=P,
                               flags=rqb_lib.RQB_FLAG_SKIP_INNER_ORTH)
    assert rc == rqb_lib.RQB_OK and kk == k == ro.k
    nA = np.linalg.norm(A)
    if dtype == torch.float64:
        assert abs(resid(A, Q, B) - resid(A, ro.Q, ro.B)) <= 1e-9 * resid(A, ro.Q, ro.B)
        assert orth_err(Q) <= 1e-12
    else:
        assert abs(resid(A, Q, B) - resid(A, ro.Q, ro.B)) <= 1e-5 * nA
        assert orth_err(Q) <= 1e-5
    # blocked: skipping the inner orth loses nothing against Fig. randQB_pb (Sec. 6.3)
    rf = orc.randqb_b(A, 0.0, b, seed=3, max_rank=k, fixed_rank=True, power=P, omega_prec=prec)
    assert abs(resid(A, Q, B) - resid(A, rf.Q, rf.B)) <= 1e-3 * resid(A, rf.Q, rf.B)


def test_power_scheme_without_inner_orth_adaptive(orc, rqb_lib):
    m, n, b = 900, 600, 40
    s = (1.0 + np.arange(n)) ** -1.0
    A = inputs.usv(m, n, s, seed=80)
    eps = 5e-2 * np.linalg.norm(A)
    ro = orc.randqb_b(A, eps, b, seed=1, power=1, skip_inner_orth=True)
    Q, B, k, rc, st = _factor(rqb_lib, A, eps, b, torch.float64, seed=1, power=1,
                              flags=rqb_lib.RQB_FLAG_SKIP_INNER_ORTH)
    assert rc == rqb_lib.RQB_OK
    check_rank(k, ro, eps, b, rel_band=1e-6)
    ro = oracle_at_rank(orc, A, ro, k, b, 1, power=1, skip_inner_orth=True)
    assert abs(resid(A, Q, B) - resid(A, ro.Q, ro.B)) <= 1e-9 * resid(A, ro.Q, ro.B)
    assert orth_err(Q) <= 1e-12


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_norm_within_tolerance_gives_empty_factorization(orc, rqb_lib, dtype):
    """||A||_F <= eps before any block (A = 0 included): k = 0 and RQB_OK, as
    the oracle; a larger A with the same eps still factors."""
    Q, B, k, rc, st = _factor(rqb_lib, np.zeros((300, 200)), 0.0, 32, dtype)
    assert rc == rqb_lib.RQB_OK and k == 0
    rng = np.random.default_rng(4)
    A = rng.standard_normal((300, 200))
    nA = np.linalg.norm(A)
    Q, B, k, rc, st = _factor(rqb_lib, A, 1.01 * nA, 32, dtype)
    assert rc == rqb_lib.RQB_OK and k == 0 == orc.randqb_b(A, 1.01 * nA, 32).k


def test_device_allocation_failure_reports_oom_and_recovers(orc, rqb_lib):
    """Host-side failure injection (rqb_inject_alloc_failure): a device
    allocation that fails makes rqb_create or rqb_factor return RQB_ERR_OOM,
    the status is recorded on the handle, and the same handle factors
    correctly on the next call."""
    A = inputs.usv(700, 500, 0.9 ** np.arange(500), seed=31).astype(np.float32).astype(np.float64)
    eps = 1e-3 * np.linalg.norm(A)
    Ad = to_dev(A, torch.float32)
    L = rqb_lib.lib()
    try:
        assert L.rqb_inject_alloc_failure(0) == rqb_lib.RQB_OK
        with pytest.raises(rqb_lib.RqbError) as e:
            rqb_lib.Handle(torch.float32)
        assert e.value.status == rqb_lib.RQB_ERR_OOM
        with rqb_lib.Handle(torch.float32) as h:
            assert L.rqb_inject_alloc_failure(0) == rqb_lib.RQB_OK
            _, _, _, rc = h.rqb_factor(Ad, eps, 32, 0, check=False)
            assert rc == rqb_lib.RQB_ERR_OOM
            assert h.rqb_get_stats().status == rqb_lib.RQB_ERR_OOM
            Q, B, k, rc = h.rqb_factor(Ad, eps, 32, 0, check=False)
            assert rc == rqb_lib.RQB_OK
            Qn, Bn = to_np(Q), to_np(B)
        ro = orc.randqb_b(A, eps, 32, seed=0, omega_prec=32)
        assert k == ro.k
        assert abs(resid(A, Qn, Bn) - resid(A, ro.Q, ro.B)) <= 1e-5 * np.linalg.norm(A)
        assert L.rqb_inject_alloc_failure(-2) == rqb_lib.RQB_ERR_INVALID
    finally:
        L.rqb_inject_alloc_failure(-1)
