"""Low-rank SVD from the factorization (rqb_svd, Sec. 2 "Computing the low rank
SVD") against the oracle's rsvd on its own factorization of the same matrix.

The GPU takes B's SVD from G = B B^T (FP64 sums of exact products) by FP64
Jacobi rotations; the oracle by one-sided Jacobi on B^T, so the two share no
method.  Checks:
  S      |S_gpu - S_orc| <= tol sigma_1 (tol 1e-5 FP32 / 1e-11 FP64: the
         factorizations agree to that, and singular values move at most by
         the perturbation of B, Weyl)
  U, Vt  U orthonormal (1e-5 / 1e-12); U diag(S) Vt rebuilds Q B of the same
         handle; the rank-r truncation error equals sqrt(sum_{i>r} S_i^2)
         (Eckart-Young on B); the leading singular subspaces agree with the
         oracle's where the gaps are wide
  known  S_i <= s_i (interlacing, B = Q^T A) and the leading S_i equal the
         planted s_i
"""
import numpy as np
import pytest
import torch

import inputs
from parity_util import orth_err, to_dev, to_np

pytestmark = pytest.mark.gpu


def _f32(x):
    return x.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("m,n,b,rate,rel_eps", [(1500, 1000, 64, 60, 1e-3), (3000, 2000, 128, 100, 1e-3),
                                                (700, 900, 50, 30, 1e-2)])
def test_svd_fp32_matches_oracle(orc, rqb_lib, m, n, b, rate, rel_eps):
    s = inputs.spectrum_exp(min(m, n), rate)
    A = _f32(inputs.usv(m, n, s, seed=m + n))
    eps = rel_eps * np.linalg.norm(A)
    with rqb_lib.Handle(torch.float32) as h:
        Qd, Bd, k, rc = h.rqb_factor(to_dev(A, torch.float32), eps, b, 3)
        Q, B = to_np(Qd), to_np(Bd)
        U, S, Vt, sweeps = h.rqb_svd(k)
        U, Vt = to_np(U), to_np(Vt)
    ro = orc.randqb_b(A, eps, b, seed=3, omega_prec=32)
    assert ro.k == k
    Uo, So, Vto = orc.rsvd(ro.Q, ro.B, k)
    print("k", k, "sweeps", sweeps, "max |dS|/s1", np.max(np.abs(S - So)) / So[0])
    assert np.all(np.diff(S) <= 0)
    assert np.max(np.abs(S - So)) <= 1e-5 * So[0]
    assert orth_err(U) <= 1e-5
    QB = Q @ B
    assert np.linalg.norm((U * S) @ Vt - QB) <= 1e-5 * np.linalg.norm(QB)
    assert np.all(S <= s[:k] * (1 + 1e-5))
    assert np.allclose(S[:k // 4], s[:k // 4], rtol=1e-4)
    for r in (k // 3, k - 1):
        e = np.linalg.norm(QB - (U[:, :r] * S[:r]) @ Vt[:r])
        assert abs(e - np.sqrt(np.sum(S[r:] ** 2))) <= 1e-5 * np.linalg.norm(QB)
    # leading subspace (well separated for this spectrum): projectors agree
    r = 8
    assert np.abs(U[:, :r] @ U[:, :r].T - Uo[:, :r] @ Uo[:, :r].T).max() <= 1e-4


def test_svd_fp64_config1(orc, rqb_lib):
    A, cfg = inputs.config_fp64(seed=1)
    eps, b = cfg["eps"], cfg["b"]
    with rqb_lib.Handle(torch.float64) as h:
        Qd, Bd, k, rc = h.rqb_factor(to_dev(A), eps, b, 0)
        Q, B = to_np(Qd), to_np(Bd)
        U, S, Vt, sweeps = h.rqb_svd(k)
        U, Vt = to_np(U), to_np(Vt)
    ro = orc.randqb_b(A, eps, b, seed=0)
    assert ro.k == k
    _, So, _ = orc.rsvd(ro.Q, ro.B, k)
    print("fp64 k", k, "sweeps", sweeps, "max |dS|/s1", np.max(np.abs(S - So)) / So[0])
    assert np.max(np.abs(S - So)) <= 1e-11 * So[0]
    assert orth_err(U) <= 1e-12
    assert np.linalg.norm((U * S) @ Vt - Q @ B) <= 1e-12 * np.linalg.norm(B)


def test_svd_odd_rank_and_truncated(orc, rqb_lib):
    """k odd (the Jacobi index set is padded by one) and r < k."""
    m, n = 1200, 800
    s = inputs.spectrum_poly(min(m, n), 1.0)
    A = _f32(inputs.usv(m, n, s, seed=7))
    with rqb_lib.Handle(torch.float32, max_rank=333, fixed_rank=True) as h:
        Qd, Bd, k, rc = h.rqb_factor(to_dev(A, torch.float32), 0.0, 64, 5)
        assert k == 333
        Q, B = to_np(Qd), to_np(Bd)
        U, S, Vt, _ = h.rqb_svd(100)
        U, Vt = to_np(U), to_np(Vt)
    assert U.shape == (m, 100) and Vt.shape == (100, n) and S.shape == (100,)
    sv = np.linalg.svd(B, compute_uv=False)     # property: the singular values of the handle's own B
    assert np.max(np.abs(S - sv[:100])) <= 1e-5 * sv[0]
    assert orth_err(U) <= 1e-5 and orth_err(Vt[:50].T) <= 1e-4


def test_svd_invalid(rqb_lib):
    with rqb_lib.Handle(torch.float32) as h:
        with pytest.raises(rqb_lib.RqbError):
            h._last_shape = (10, 10)
            h.rqb_svd(3)              # no factorization on the handle
        A = torch.randn(400, 300, device="cuda").t().contiguous().t()
        _, _, k, _ = h.rqb_factor(A, 0.5 * float(A.norm()), 32, 0)
        with pytest.raises(rqb_lib.RqbError):
            h.rqb_svd(k + 1)


def test_svd_bf16_handle(orc, rqb_lib):
    """BF16 storage handle: Q and B are FP32, so rqb_svd runs as for FP32; its
    leading singular values match the planted spectrum to the BF16 storage
    level and the factors rebuild the handle's own Q B."""
    m, n, b = 2048, 1300, 128
    s = inputs.spectrum_exp(min(m, n), 150)
    A = orc.round_bf16_array(inputs.usv(m, n, s, seed=m + n))
    eps = 1e-2 * np.linalg.norm(A)
    with rqb_lib.Handle(torch.bfloat16) as h:
        Qd, Bd, k, rc = h.rqb_factor(to_dev(A, torch.bfloat16), eps, b, 3)
        assert rc == rqb_lib.RQB_OK
        Q, B = to_np(Qd), to_np(Bd)
        U, S, Vt, _ = h.rqb_svd(k)
        U, Vt = to_np(U), to_np(Vt)
    sv = np.linalg.svd(A, compute_uv=False)
    assert orth_err(U) <= 1e-5
    QB = Q @ B
    assert np.linalg.norm((U * S) @ Vt - QB) <= 1e-5 * np.linalg.norm(QB)
    # top singular values: BF16 residual roundings perturb them by ~2^-9 sigma_1
    assert np.all(np.abs(S[:k // 4] - sv[:k // 4]) <= 2.0 ** -8 * sv[0])
