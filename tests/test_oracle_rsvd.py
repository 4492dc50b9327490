"""Pins of the oracle's low-rank SVD from a QB factorization (Sec. 2, computing
the low rank SVD: the SVD of B gives A ~ Q B = (Q Uh) D Vh^T).

Fixed by the mathematics: for B = U0 diag(s0) V0^T with known s0 the factors
reproduce s0, are orthonormal and rebuild Q B; truncation to r leaves exactly
the Eckart-Young error (sum of the dropped s0_i^2); the singular values agree
with LAPACK's (numpy); a zero singular value gives a zero row of Vt.
"""
import numpy as np
import pytest

import inputs


def _case(m, k, n, s0, seed):
    rng = np.random.default_rng(seed)
    Q = inputs.haar_factor(m, k, rng)
    U0 = inputs.haar_factor(k, k, rng)
    V0 = inputs.haar_factor(n, k, rng)
    B = (U0 * s0) @ V0.T
    return Q, B


@pytest.mark.parametrize("m,k,n", [(60, 12, 40), (90, 31, 31), (200, 7, 300)])
def test_rsvd_known_spectrum(orc, m, k, n):
    s0 = np.sort(np.exp(-np.arange(k) / 3.0) * 2.0)[::-1]
    Q, B = _case(m, k, n, s0, m + k + n)
    U, S, Vt = orc.rsvd(Q, B, k)
    assert np.allclose(S, s0, rtol=1e-12, atol=0)
    assert np.abs(U.T @ U - np.eye(k)).max() <= 1e-12
    assert np.abs(Vt @ Vt.T - np.eye(k)).max() <= 1e-12
    assert np.linalg.norm((U * S) @ Vt - Q @ B) <= 1e-12 * np.linalg.norm(B)


def test_rsvd_truncation_is_eckart_young(orc):
    k = 20
    s0 = np.linspace(3.0, 0.1, k)
    Q, B = _case(80, k, 50, s0, 3)
    for r in (1, 5, 19):
        U, S, Vt = orc.rsvd(Q, B, r)
        err2 = np.linalg.norm(Q @ B - (U * S) @ Vt) ** 2
        assert abs(err2 - np.sum(s0[r:] ** 2)) <= 1e-12 * np.sum(s0 ** 2)
        # basis-free: the projector onto the leading left singular space
        ul = np.linalg.svd(B)[0][:, :r]
        P = Q @ ul
        assert np.abs(U @ U.T - P @ P.T).max() <= 1e-10


def test_rsvd_matches_lapack_values(orc):
    rng = np.random.default_rng(9)
    B = rng.standard_normal((25, 70))
    Q = inputs.haar_factor(100, 25, rng)
    _, S, _ = orc.rsvd(Q, B, 25)
    assert np.allclose(S, np.linalg.svd(B, compute_uv=False), rtol=1e-12)


def test_rsvd_zero_singular_value(orc):
    s0 = np.array([2.0, 1.0, 0.5, 0.0])
    Q, B = _case(30, 4, 12, s0, 5)     # rank 3
    U, S, Vt = orc.rsvd(Q, B, 4)
    assert S[3] <= 1e-14 and np.allclose(S[:3], s0[:3], rtol=1e-12)
    assert np.abs(U.T @ U - np.eye(4)).max() <= 1e-12
    assert np.linalg.norm((U * S) @ Vt - Q @ B) <= 1e-12 * np.linalg.norm(B)


def test_rsvd_rejects_bad_rank(orc):
    Q, B = _case(20, 5, 10, np.ones(5), 1)
    with pytest.raises(ValueError):
        orc.rsvd(Q, B, 6)
