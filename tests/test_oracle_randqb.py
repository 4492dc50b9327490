"""Pins of the oracle's randQB_b / randQB_pb against what the paper and the
mathematics fix, independently of the oracle's own code:

  Prop. 4.1(a)  Q orthonormal                                  (Sec. 4.1)
  Prop. 4.1(b)  A^(i) = (I - Q Q^T) A and B = Q^T A, recomputed with numpy
  Sec. 4.2      E_i = ||A||^2 - sum ||B_j||^2 equals the direct ||A^(i)||^2
  Sec. 4.1      blocked and unblocked projectors coincide for one Omega,
                the unblocked one from LAPACK's QR of A Omega
  eq. minerrors / Eckart-Young: the residual is never below the SVD tail, and
                k is at least the optimal eps-rank
  Algorithm 1 with (4a)-(4c): b = 1 is the greedy single-vector scheme,
                written out below in numpy
  exact rank r <= b: one block, zero residual
  orthogonal invariance, fixed-rank mode (Sec. 4.1), rank cap
  Fig. randQB_pb: the power scheme never does worse than P = 0 at fixed rank
  Sec. 6.2 golden: Matrix 1 has rank about 75 at precision 1e-15
  Sec. 5.4 / 6.3 golden: the unblocked power scheme without re-orthonormalisation
                stalls near sigma_1 eps_mach^(1/(2P+1)); the blocked one does not.
"""
import json
import os

import numpy as np
import pytest

import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tail(s, k):
    return float(np.sqrt(np.sum(s[k:] ** 2)))


def _eps_rank(s, eps):
    """smallest k with sqrt(sum_{j>k} s_j^2) <= eps (eq. minerrors)."""
    t = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])  # t[k] = tail from index k
    t = np.append(t, 0.0)
    return int(np.argmax(t <= eps))


@pytest.fixture(scope="module")
def case_fp64():
    A, meta = inputs.config_fp64()
    return A, meta


@pytest.fixture(scope="module")
def res_fp64(orc, case_fp64):
    A, meta = case_fp64
    return orc.randqb_b(A, meta["eps"], meta["b"], seed=0)


def test_prop41a_orthonormal(res_fp64):
    Q = res_fp64.Q
    assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-12


def test_prop41b_B_equals_QtA_and_residual(res_fp64, case_fp64):
    A, _ = case_fp64
    Q, B = res_fp64.Q, res_fp64.B
    nA = np.linalg.norm(A)
    assert np.abs(Q.T @ A - B).max() < 1e-12 * nA
    R = A - Q @ B
    R2 = A - Q @ (Q.T @ A)
    assert np.linalg.norm(R - R2) < 1e-12 * nA
    # per-block: D_i = ||A - Qbar_i Qbar_i^T A||^2
    b = 50
    for i in range(res_fp64.blocks):
        Qi = Q[:, :(i + 1) * b]
        d = np.linalg.norm(A - Qi @ (Qi.T @ A)) ** 2
        assert abs(d - res_fp64.D[i]) < 1e-12 * nA ** 2


def test_downdate_equals_direct(res_fp64, case_fp64):
    A, _ = case_fp64
    nA2 = np.linalg.norm(A) ** 2
    assert abs(res_fp64.normA2 - nA2) < 1e-13 * nA2
    assert np.all(np.abs(res_fp64.E - res_fp64.D) < 64 * np.finfo(float).eps * nA2)
    # ||A - QB||^2 = ||A||^2 - ||B||^2 (Prop. 4.1(b) with Pythagoras)
    nB2 = np.linalg.norm(res_fp64.B) ** 2
    assert abs(res_fp64.E[-1] - (nA2 - nB2)) < 64 * np.finfo(float).eps * nA2


def test_eckart_young_and_rank_recovery(res_fp64, case_fp64):
    A, meta = case_fp64
    s = meta["sigma"]
    k = res_fp64.k
    resid = np.linalg.norm(A - res_fp64.Q @ res_fp64.B)
    assert resid <= meta["eps"]
    assert resid >= _tail(s, k) * (1 - 1e-6)
    kopt = _eps_rank(s, meta["eps"])
    b = meta["b"]
    assert kopt <= k <= int(np.ceil(kopt / b)) * b + 2 * b
    assert res_fp64.status == 0
    assert res_fp64.k % b == 0


def test_eckart_young_small_brute_force_svd(orc):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((30, 20)) @ np.diag(0.7 ** np.arange(20)) @ rng.standard_normal((20, 20))
    s = orc.svd_values(A)
    sn = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, sn, rtol=1e-10)
    for eps_rel in (1e-1, 1e-2, 1e-4):
        eps = eps_rel * np.linalg.norm(A)
        r = orc.randqb_b(A, eps, 3, seed=2)
        resid = np.linalg.norm(A - r.Q @ r.B)
        assert resid <= eps * (1 + 1e-12)
        assert resid >= _tail(s, r.k) * (1 - 1e-9)
        assert r.k >= _eps_rank(s, eps)


def test_blocked_projector_equals_unblocked(orc):
    """Sec. 4.1: for one Omega, blocked and unblocked QQ^T are the projector onto R(A Omega)."""
    rng = np.random.default_rng(8)
    m, n, k, b = 300, 200, 50, 10
    s = 0.9 ** np.arange(n)
    A = inputs.usv(m, n, s, seed=21)
    r = orc.randqb_b(A, 0.0, b, seed=17, max_rank=k, fixed_rank=True)
    assert r.k == k
    Om = orc.omega(seed=17, n=n, col0=0, ncols=k)
    Qt, _ = np.linalg.qr(A @ Om)
    P1 = r.Q @ r.Q.T
    P2 = Qt @ Qt.T
    assert np.linalg.norm(P1 - P2) < 1e-9
    Qu, Bu = orc.randqb(A, k, seed=17)
    assert np.linalg.norm(Qu @ Qu.T - P1) < 1e-9
    assert abs(np.linalg.norm(A - Qu @ Bu) - np.linalg.norm(A - r.Q @ r.B)) < 1e-10 * np.linalg.norm(A)
    del rng


def _algorithm1(A, eps, omegas):
    """Algorithm 1 (Sec. 1.2) with the random choice (4a)-(4c), in numpy."""
    Aj = A.copy()
    qs, bs = [], []
    j = 0
    while np.linalg.norm(Aj) > eps:
        y = Aj @ omegas[:, j]                # (4b)
        q = y / np.linalg.norm(y)            # (4c)
        bj = q @ Aj                          # (5)
        Aj = Aj - np.outer(q, bj)            # (8)
        qs.append(q)
        bs.append(bj)
        j += 1
    return np.array(qs).T, np.array(bs), j


def test_b1_is_algorithm1(orc):
    m, n = 60, 40
    s = 0.8 ** np.arange(n)
    A = inputs.usv(m, n, s, seed=31)
    eps = 1e-3 * np.linalg.norm(A)
    Om = orc.omega(seed=5, n=n, col0=0, ncols=n)
    Qa, Ba, ka = _algorithm1(A, eps, Om)
    r = orc.randqb_b(A, eps, 1, seed=5)
    assert r.k == ka
    assert np.abs(r.Q - Qa).max() < 1e-8
    assert np.abs(r.B - Ba).max() < 1e-8 * np.linalg.norm(A)


def test_exact_rank_stops_after_one_block(orc):
    m, n, rank, b = 120, 90, 7, 10
    A = inputs.usv(m, n, np.arange(rank, 0, -1).astype(float), seed=41)
    nA = np.linalg.norm(A)
    r = orc.randqb_b(A, 1e-10 * nA, b, seed=3)
    assert r.blocks == 1 and r.k == b
    assert np.linalg.norm(A - r.Q @ r.B) < 1e-13 * nA
    assert np.abs(r.Q.T @ r.Q - np.eye(b)).max() < 1e-12


def test_orthogonal_invariance(orc):
    rng = np.random.default_rng(12)
    m, n, b = 80, 50, 8
    A = inputs.usv(m, n, 0.85 ** np.arange(n), seed=51)
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    eps = 1e-4 * np.linalg.norm(A)
    r1 = orc.randqb_b(A, eps, b, seed=9)
    r2 = orc.randqb_b(U @ A, eps, b, seed=9)
    assert r1.k == r2.k
    assert np.abs(r2.Q - U @ r1.Q).max() < 1e-11
    assert np.abs(r2.B - r1.B).max() < 1e-11 * np.linalg.norm(A)


def test_fixed_rank_and_shrunk_last_block(orc):
    A = inputs.usv(70, 60, 0.9 ** np.arange(60), seed=61)
    r = orc.randqb_b(A, 1.0e9, 8, seed=1, max_rank=36, fixed_rank=True)
    assert r.k == 36 and r.blocks == 5  # 8+8+8+8+4
    assert r.status == 0
    assert np.abs(r.Q.T @ r.Q - np.eye(36)).max() < 1e-12


def test_rank_cap_full_rank(orc):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((40, 30))
    r = orc.randqb_b(A, 0.0, 7, seed=4)
    assert r.k == 30 and r.blocks == 5  # 7*4 + 2
    assert np.linalg.norm(A - r.Q @ r.B) < 1e-13 * np.linalg.norm(A)
    assert r.status in (0, 1)


def test_not_converged_status(orc):
    A = inputs.usv(50, 40, 0.95 ** np.arange(40), seed=71)
    r = orc.randqb_b(A, 1e-12, 5, seed=1, max_rank=20)
    assert r.k == 20 and r.status == 1


def test_power_scheme_never_worse(orc):
    m, n = 200, 150
    s = (1.0 + 200.0 * np.arange(n)) ** -0.5  # Matrix 2 spectrum (Sec. 6.2)
    A = inputs.usv(m, n, s, seed=81)
    errs = []
    for P in (0, 1, 2):
        r = orc.randqb_b(A, 0.0, 10, seed=6, max_rank=40, fixed_rank=True, power=P)
        assert np.abs(r.Q.T @ r.Q - np.eye(40)).max() < 1e-12
        assert np.abs(r.Q.T @ A - r.B).max() < 1e-12
        errs.append(np.linalg.norm(A - r.Q @ r.B))
    opt = _tail(s, 40)
    assert errs[0] > errs[1] > errs[2] >= opt * (1 - 1e-9)
    # Sec. 6.2: with P >= 1 the Frobenius error is essentially optimal
    assert errs[1] < 1.10 * opt and errs[2] < 1.05 * opt


def test_golden_matrix1_rank_about_75(orc):
    g = json.load(open(os.path.join(GOLDEN, "matrix1_rank.json")))
    m, n = g["paper_size"]
    A, d = inputs.matrix1(m, n, beta=g["beta"])
    # rank to the stated precision, from the known singular values
    rank = int(np.sum(d > g["precision"]))
    assert abs(rank - g["rank_about"]) <= g["band"]
    # the oracle's blocked scheme recovers it to within a block or two
    nA = np.linalg.norm(A)
    eps = 1e-7 * nA   # stop rule resolves down to ~sqrt(u) ||A|| (FP64 downdate)
    r = orc.randqb_b(A, eps, g["paper_block_size"], seed=0)
    kopt = _eps_rank(np.sort(d)[::-1], eps)
    assert kopt <= r.k <= kopt + 2 * g["paper_block_size"]
    # at fixed rank rank+b the residual reaches the precision the paper states
    r2 = orc.randqb_b(A, 0.0, g["paper_block_size"], seed=0, max_rank=rank + 10, fixed_rank=True)
    assert np.linalg.norm(A - r2.Q @ r2.B) < 20 * g["precision"]


def test_golden_unblocked_power_floor_vs_blocked(orc):
    g = json.load(open(os.path.join(GOLDEN, "unblocked_power_floor.json")))
    m, n = 300, 200
    d = 0.7 ** np.arange(n)      # sigma_1 = 1, fast decay far below the floors
    A = inputs.usv(m, n, d, seed=91)
    k = 70                        # 0.7^70 ~ 1.4e-11
    u = np.finfo(float).eps
    for P in (1, 2):
        # unblocked (one block of width k) without re-orthonormalisation, Sec. 5.4
        ru = orc.randqb_b(A, 0.0, k, seed=3, max_rank=k, fixed_rank=True, power=P, skip_inner_orth=True)
        eu = np.linalg.norm(A - ru.Q @ ru.B)
        # blocked, same skip
        rb = orc.randqb_b(A, 0.0, 10, seed=3, max_rank=k, fixed_rank=True, power=P, skip_inner_orth=True)
        eb = np.linalg.norm(A - rb.Q @ rb.B)
        floor_here = u ** (1.0 / (2 * P + 1))      # same law at this machine's epsilon
        assert eu > 0.01 * floor_here              # unblocked stalls near the floor
        assert eb < 1e-8                           # blocked reaches full precision
        assert eb < 1e-3 * eu
    assert g["floor"]["1"] == 1e-5 and g["floor"]["2"] == 1e-3


def test_norm_within_tolerance_gives_empty_factorization(orc):
    """||A||_F <= eps before any block: k = 0 meets the tolerance (A = 0 included,
    whose sketch has no orthonormal basis)."""
    A = np.zeros((50, 40))
    r = orc.randqb_b(A, 0.0, 8, seed=1)
    assert r.k == 0 and r.blocks == 0 and r.status == 0
    rng = np.random.default_rng(3)
    A = 1e-3 * rng.standard_normal((60, 30))
    nA = np.linalg.norm(A)
    r = orc.randqb_b(A, 1.01 * nA, 8, seed=1)
    assert r.k == 0 and r.status == 0
    r = orc.randqb_b(A, 0.5 * nA, 8, seed=1)
    assert r.k >= 8 and r.status == 0
