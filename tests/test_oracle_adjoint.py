"""Pin of the oracle's gradient through the fixed-rank map X = Q Q^T A
(Q = orth(A Omega), Omega fixed).  The paper has no derivatives; the formula
dA = Q Q^T G + (I - Q Q^T)(G B^T + A G^T Q) R^{-T} Omega^T, R = B Omega, comes
from differentiating the projector onto R(A Omega) (Sec. 4.1, Prop. 4.1(c)).
It is checked against FP64 central finite differences (h = 1e-6) of the
oracle's own forward map, on a 256 x 128 instance of the adjoint workload's
construction (N(0,1)/sqrt(n) plus a planted low-rank part of norm 10)."""
import math

import numpy as np
import pytest

import inputs


def _instance():
    A, T, _ = inputs.config_adjoint_np(m=256, n=128, seed=55, rank=16, norm=10.0)
    return A, T


def _loss_and_grad(orc, A, T, k, b, seed):
    r = orc.randqb_b(A, 0.0, b, seed=seed, max_rank=k, fixed_rank=True)
    X = r.Q @ r.B
    L = float(np.sum((X - T) ** 2))
    G = 2.0 * (X - T)
    return L, r, G


@pytest.mark.parametrize("k,b", [(32, 8), (48, 16)])
def test_adjoint_matches_central_differences(orc, k, b):
    A, T = _instance()
    L, r, G = _loss_and_grad(orc, A, T, k, b, seed=4)
    dA = orc.qqta_adjoint(A, r.Q, r.B, G, seed=4)
    rng = np.random.default_rng(9)
    h = 1e-6
    for trial in range(6):
        V = rng.standard_normal(A.shape)
        V /= np.linalg.norm(V)
        Lp = _loss_and_grad(orc, A + h * V, T, k, b, 4)[0]
        Lm = _loss_and_grad(orc, A - h * V, T, k, b, 4)[0]
        fd = (Lp - Lm) / (2 * h)
        an = float(np.sum(dA * V))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-7 * np.linalg.norm(dA), (trial, fd, an)
    # single entries, including ones in the planted low-rank part's support
    for (i, j) in [(0, 0), (17, 3), (255, 127), (100, 64)]:
        E = np.zeros_like(A)
        E[i, j] = 1.0
        fd = (_loss_and_grad(orc, A + h * E, T, k, b, 4)[0] - _loss_and_grad(orc, A - h * E, T, k, b, 4)[0]) / (2 * h)
        assert abs(fd - dA[i, j]) <= 1e-5 * max(1.0, abs(dA[i, j])), (i, j, fd, dA[i, j])


def test_adjoint_is_projection_gradient_for_full_rank(orc):
    """k = n: Q Q^T A = A for every A, so X = A and dL/dA = G exactly."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 24))
    T = rng.standard_normal((40, 24))
    L, r, G = _loss_and_grad(orc, A, T, 24, 8, 1)
    dA = orc.qqta_adjoint(A, r.Q, r.B, G, seed=1)
    assert np.abs(dA - G).max() <= 1e-9 * np.abs(G).max()
