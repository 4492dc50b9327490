"""Pins of the oracle's orth() (Sec. 2.4: thin unpivoted QR, diag(R) >= 0) and of
its singular-value routine (used for the Eckart-Young bound, eq. minerrors)."""
import numpy as np
import pytest


def _lapack_q(Y):
    Qn, Rn = np.linalg.qr(Y, mode="reduced")
    s = np.sign(np.diag(Rn))
    s[s == 0] = 1
    return Qn * s, (Rn.T * s).T


@pytest.mark.parametrize("m,p", [(50, 20), (300, 64), (64, 64), (1000, 3), (7, 1)])
def test_orth_matches_lapack_householder(orc, m, p):
    rng = np.random.default_rng(m * 1000 + p)
    Y = rng.standard_normal((m, p))
    Q, R = orc.orth(Y, return_r=True)
    Qn, Rn = _lapack_q(Y)
    assert np.abs(Q - Qn).max() < 1e-12
    assert np.abs(R - Rn).max() < 1e-12 * np.abs(Rn).max()
    assert np.abs(Q.T @ Q - np.eye(p)).max() < 1e-14 * max(10, p)
    assert np.abs(Q @ R - Y).max() < 1e-13 * np.abs(Y).max() * np.sqrt(m)
    assert np.all(np.diag(R) > 0)
    assert np.abs(np.tril(R, -1)).max() == 0.0


def test_orth_rank_deficient_still_orthonormal(orc):
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((40, 6))
    Y[:, 2] = 0.0
    Y[:, 4] = Y[:, 0] * 2.0  # dependent column
    Q, R = orc.orth(Y, return_r=True)
    assert np.abs(Q.T @ Q - np.eye(6)).max() < 1e-13
    assert np.abs(Q @ R - Y).max() < 1e-13
    assert np.all(np.diag(R) >= 0)
    assert R[2, 2] == 0.0


@pytest.mark.parametrize("m,n", [(40, 30), (30, 40), (25, 25), (60, 1)])
def test_svd_values_match_lapack(orc, m, n):
    rng = np.random.default_rng(m + 7 * n)
    A = rng.standard_normal((m, n)) @ np.diag(np.logspace(0, -6, n))
    s = orc.svd_values(A)
    sn = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, sn, rtol=1e-10, atol=1e-14 * sn[0])
