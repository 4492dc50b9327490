"""Pins of the oracle's BF16 modes (the BF16 storage leg of the precision form).

round_bf16: 8 significant bits, nearest, ties to even (fixed by the format).
omega prec 8: the binary32 draw of Fig. randQB_b line (2) rounded to BF16.
storage_prec 16: the residual A^(i) is rounded to BF16 after every downdate
(line (5)) and the stop test is the stored residual's direct norm (line (6)).
With W_i = rnd(W_{i-1} - Q_i B_i) = W_{i-1} - Q_i B_i + E_i, the factors satisfy
A - Q B = W_s - sum_i E_i exactly, and |E_i| <= 2^-9 |W_{i-1} - Q_i B_i| entrywise,
which bounds the gap between the true residual and the stored one.
"""
import numpy as np
import pytest

import inputs


def test_round_bf16_closed_forms(orc):
    r = orc.round_bf16
    u = 2.0 ** -7                         # BF16 spacing on [1, 2)
    assert r(1.0) == 1.0 and r(0.0) == 0.0 and r(-6.0) == -6.0
    assert r(1.0 + u / 2) == 1.0          # tie -> even (mantissa 0)
    assert r(1.0 + 3 * u / 2) == 1.0 + 2 * u   # tie -> even (mantissa 2)
    assert r(-(1.0 + 3 * u / 2)) == -(1.0 + 2 * u)
    assert r(1.0 + u / 4) == 1.0 and r(1.0 + 3 * u / 4) == 1.0 + u
    assert r(2.0 - u / 4) == 2.0          # carry into the next binade
    assert r(3.0 * 2.0 ** -100) == 3.0 * 2.0 ** -100


def test_omega_bf16_is_rounded_binary32_draw(orc):
    a = orc.omega(seed=7, n=3000, col0=0, ncols=64, prec=32)
    b = orc.omega(seed=7, n=3000, col0=0, ncols=64, prec=8)
    nz = a != 0
    e = np.floor(np.log2(np.abs(a[nz]))) + 1
    assert np.all(np.abs(b[nz] - a[nz]) <= 2.0 ** (e - 9) * (1 + 1e-12))
    scaled = b[nz] * 2.0 ** (8 - e)
    assert np.all((np.abs(scaled - np.round(scaled)) == 0) | (np.abs(b[nz]) == 2.0 ** e))
    x = b.ravel()
    assert abs(x.mean()) < 5 / np.sqrt(x.size) and abs(x.var() - 1.0) < 0.01


def _bf16(x):
    import torch
    return torch.as_tensor(x, dtype=torch.float32).to(torch.bfloat16).double().numpy()


@pytest.mark.parametrize("m,n,b,rate,rel_eps", [(600, 400, 32, 40, 1e-2), (500, 450, 50, 80, 2e-2)])
def test_bf16_storage_factorization(orc, m, n, b, rate, rel_eps):
    A = _bf16(inputs.usv(m, n, inputs.spectrum_exp(min(m, n), rate), seed=m + n))
    nA = np.linalg.norm(A)
    eps = rel_eps * nA
    r = orc.randqb_b(A, eps, b, seed=3, omega_prec=8, storage_prec=16)
    assert r.status == 0
    assert np.abs(r.Q.T @ r.Q - np.eye(r.k)).max() <= 1e-12            # Prop. 4.1(a)
    assert r.D[-1] <= eps * eps                                         # line (6) on the stored residual
    assert np.all(np.diff(r.D) < 0)
    # A - Q B = W_s - sum E_i: the true residual is within sum ||E_i|| of the stored one
    true_res = np.linalg.norm(A - r.Q @ r.B)
    bound = 2.0 ** -9 * (nA + np.sum(np.sqrt(r.D[:-1]))) * 1.01
    assert abs(true_res - np.sqrt(r.D[-1])) <= bound
    # the unrounded oracle reaches a rank at most one block away
    r64 = orc.randqb_b(A, eps, b, seed=3, omega_prec=8)
    assert abs(r.k - r64.k) <= b


def test_storage_64_is_plain_oracle(orc):
    A = inputs.usv(300, 200, inputs.spectrum_exp(200, 20), seed=5)
    a = orc.randqb_b(A, 1e-3 * np.linalg.norm(A), 20, seed=1)
    c = orc.randqb_b(A, 1e-3 * np.linalg.norm(A), 20, seed=1, storage_prec=64)
    assert a.k == c.k and np.array_equal(a.Q, c.Q) and np.array_equal(a.B, c.B)


def test_round_bf16_array_matches_scalar(orc):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((37, 11)) * 10.0 ** rng.integers(-30, 30, size=(37, 11))
    x[0, 0], x[1, 0], x[2, 0] = 1.0 + 2.0 ** -8, -(1.0 + 3 * 2.0 ** -8), 0.0
    y = orc.round_bf16_array(x)
    assert y.shape == x.shape
    assert np.array_equal(y, np.vectorize(orc.round_bf16)(x))
    assert y[0, 0] == 1.0 and y[1, 0] == -(1.0 + 2.0 ** -6) and y[2, 0] == 0.0
