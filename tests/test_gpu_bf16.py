"""BF16 storage path (RQB_BF16 handles) against the oracle's BF16 modes.

A and the downdated residual are stored in BF16; the three products of
Fig. randQB_b that read all of A run on BF16 tensor-core MMAs with FP32
accumulation:
  line (3)  Y = W Omega_i    Omega_i the binary32 draw rounded to BF16, so the
                             products are exact and only the FP32 sums round
  line (4)  B_i = Q_i^T W    Q_i split into BF16 hi + lo (2^-18 of each value)
  line (5)  W <- rn_bf16(W - Q_i B_i), Q_i and B_i split, three passes
The oracle reproduces the model with omega_prec=8 (Omega) and storage_prec=16
(the residual rounded after every downdate, stop on the stored residual's
norm).  Tolerances:
  sketch / project   relative Frobenius error <= 2e-5 (FP32 sums; the Q split)
  downdate           entrywise |W_gpu - x| <= 2^-8 |x| + 2^-16 (|Q| |B|)_ij
                     with x = A - Q B in FP64 (one BF16 rounding of a value
                     within 2^-16 (|Q||B|)_ij of x); W_gpu equals the
                     oracle's rn_bf16(x) except at rounding ties of that size
  randQB_b           rank as the oracle's (or one block away when the oracle's
                     stored norm is within 1e-2 of eps^2, then compared with the
                     oracle rerun at the GPU's rank); ||Q^T Q - I|| <= 1e-5;
                     |  ||A - QB||_F - sqrt(D_s) | <= 1.01 2^-9 sum_i sqrt(D_i)
                     + 2e-5 sum_i sqrt(D_(i-1)) (A - QB = W_s - sum of the
                     rounding errors, each at most 2^-9 of its block's residual);
                     |r_gpu - r_oracle| within the sum of both sides' gaps and
                     of the stored-norm band
Entry by entry: the sketch within 1e-6 (|W| |Omega|)_ij of W Omega with the
handle's own Omega (exact products, FP32 sums) and within that plus
|W| |Omega_gpu - Omega_oracle| of the oracle's; the projection within
1e-5 (|Q^T| |W|)_ij (the 2^-18 split of Q plus FP32 sums).
Shapes span several 128-row tiles and 64-wide K chunks with ragged tails.
"""
import numpy as np
import pytest
import torch

import inputs
from parity_util import assert_elementwise, orth_err, product_bound, resid, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL_STEP = 2e-5


@pytest.fixture(scope="module")
def hbf(rqb_lib):
    with rqb_lib.Handle(torch.bfloat16) as h:
        yield h


def _bf(orc, x):
    """x rounded to BF16 by the oracle (float64 array of BF16 values)."""
    return orc.round_bf16_array(x)


def test_omega_is_rounded_binary32_draw(orc, hbf):
    g = to_np(hbf.rqb_omega(3000, 40, 256, seed=99))
    o = orc.omega(99, 3000, 40, 256, prec=8)
    assert np.array_equal(_bf(orc, g), g)
    diff = g != o
    assert diff.mean() < 1e-3
    assert np.all(np.abs(g - o)[diff] <= 2.0 ** -7 * np.abs(o)[diff])


@pytest.mark.parametrize("m,n,p,col0", [(1000, 700, 64, 0), (3000, 2000, 256, 128), (1037, 777, 37, 5),
                                        (129, 257, 32, 0), (4100, 300, 128, 64), (2000, 1500, 100, 3)])
def test_sketch(orc, hbf, m, n, p, col0):
    rng = np.random.default_rng(m + 3 * n + p)
    A = _bf(orc, rng.standard_normal((m, n)))
    Y, nrm = hbf.rqb_sketch(to_dev(A, torch.bfloat16), col0, p, seed=17)
    Yg = to_np(Y)
    Om = to_np(hbf.rqb_omega(n, col0, p, seed=17))
    Yh = A @ Om                                   # the handle's own Omega, FP64
    assert np.linalg.norm(Yg - Yh) <= 2e-6 * np.linalg.norm(Yh)
    Yo = orc.sketch(A, 17, col0, p, omega_prec=8)
    assert np.linalg.norm(Yg - Yo) <= TOL_STEP * np.linalg.norm(Yo)
    assert abs(nrm - np.sum(A * A)) <= 1e-9 * np.sum(A * A)
    bound = product_bound(A, Om)
    assert_elementwise(Yg, Yh, bound, 1e-6, "BF16 sketch vs W Omega_gpu")
    Oo = orc.omega(17, n, col0, p, prec=8)
    assert_elementwise(Yg, Yo, bound, 1e-6, "BF16 sketch vs oracle", extra=np.abs(A) @ np.abs(Om - Oo))


def test_sketch_unaligned_lda(orc, hbf):
    """lda not a multiple of 8: the matrix is copied to an aligned buffer first."""
    rng = np.random.default_rng(1)
    A = _bf(orc, rng.standard_normal((1001, 600)))
    Y, _ = hbf.rqb_sketch(to_dev(A, torch.bfloat16, lda=1005), 0, 50, seed=2)
    Yo = orc.sketch(A, 2, 0, 50, omega_prec=8)
    assert np.linalg.norm(to_np(Y) - Yo) <= TOL_STEP * np.linalg.norm(Yo)


@pytest.mark.parametrize("m,n,p", [(3000, 2000, 50), (1037, 777, 37), (500, 4100, 128), (2048, 1024, 256),
                                   (130, 300, 64)])
def test_project(orc, hbf, m, n, p):
    rng = np.random.default_rng(m * n + p)
    A = _bf(orc, rng.standard_normal((m, n)))
    Q = np.linalg.qr(rng.standard_normal((m, p)))[0].astype(np.float32).astype(np.float64)
    Bi, nb2 = hbf.rqb_project(to_dev(Q, torch.float32), to_dev(A, torch.bfloat16))
    Bo = Q.T @ A
    Bg = to_np(Bi)
    assert np.linalg.norm(Bg - Bo) <= TOL_STEP * np.linalg.norm(Bo)
    assert abs(nb2 - np.sum(Bg * Bg)) <= 1e-12 * np.sum(Bg * Bg)
    assert_elementwise(Bg, Bo, product_bound(Q.T, A), 1e-5, "BF16 Q^T W")


@pytest.mark.parametrize("m,n,p,ncols,inplace", [(2000, 1000, 50, 50, False), (1037, 777, 37, 37, True),
                                                 (3000, 2100, 256, 128, False), (129, 300, 64, 200, True)])
def test_downdate_sketch(orc, hbf, m, n, p, ncols, inplace):
    rng = np.random.default_rng(m + n + p)
    A = _bf(orc, rng.standard_normal((m, n)))
    Q = np.linalg.qr(rng.standard_normal((m, p)))[0].astype(np.float32).astype(np.float64)
    B = (Q.T @ A).astype(np.float32).astype(np.float64)
    Ad = to_dev(A, torch.bfloat16)
    W = Ad if inplace else to_dev(np.zeros((m, n)), torch.bfloat16)
    Y, nw2 = hbf.rqb_downdate_sketch(Ad, to_dev(Q, torch.float32), to_dev(B, torch.float32), W, 11, ncols, seed=4)
    Wg = to_np(W)
    x = A - Q @ B
    slack = 2.0 ** -16 * (np.abs(Q) @ np.abs(B))
    assert np.all(np.abs(Wg - x) <= 2.0 ** -8 * np.abs(x) + slack)
    Wo = _bf(orc, x)
    assert np.mean(Wg != Wo) < 1e-2
    # exact FP32 squares summed 32 at a time in FP32 (<= 32 2^-24 relative), then in FP64
    assert abs(nw2 - np.sum(Wg * Wg)) <= 2e-6 * np.sum(Wg * Wg)
    Om = to_np(hbf.rqb_omega(n, 11, ncols, seed=4))
    Yh = Wg @ Om
    assert np.linalg.norm(to_np(Y) - Yh) <= 2e-6 * np.linalg.norm(Yh)
    assert_elementwise(to_np(Y), Yh, product_bound(Wg, Om), 1e-6, "BF16 downdated W Omega")


def _factor(rqb, A, eps, b, seed, **kw):
    with rqb.Handle(torch.bfloat16, **kw) as h:
        Q, B, k, rc = h.rqb_factor(to_dev(A, torch.bfloat16), eps, b, seed, check=False)
        st = h.rqb_get_stats()
        return to_np(Q), to_np(B), k, rc, st


def _stored_gap_bound(D, nA2):
    """Bound on | ||A - QB||_F - sqrt(D_s) | from the BF16 roundings of the
    residual (2^-9 of each block's residual) and the split products."""
    d = np.sqrt(np.maximum(np.asarray(D), 0.0))
    prev = np.concatenate([[np.sqrt(nA2)], d[:-1]])
    return 1.01 * 2.0 ** -9 * d.sum() + 2e-5 * prev.sum()


def _check_rank_d(k, ro, eps, b):
    if k == ro.k:
        return
    e2 = eps * eps
    Ds = list(ro.D)
    cands = [Ds[-1]] + ([Ds[-2]] if len(Ds) > 1 else [])
    assert any(abs(d - e2) <= 1e-2 * e2 for d in cands) and abs(k - ro.k) <= b, \
        f"rank {k} != oracle {ro.k} (D tail {Ds[-2:]}, eps^2 {e2})"


@pytest.mark.parametrize("m,n,b,rate,rel_eps", [(1500, 1000, 64, 60, 2e-2), (2049, 1300, 128, 150, 1e-2),
                                                (1000, 1200, 50, 40, 5e-2), (4096, 2048, 256, 150, 1e-2),
                                                (700, 640, 32, 30, 2e-2)])
def test_randqb_matches_oracle(orc, rqb_lib, m, n, b, rate, rel_eps):
    s = inputs.spectrum_exp(min(m, n), rate)
    A = _bf(orc, inputs.usv(m, n, s, seed=m + n))
    nA = np.linalg.norm(A)
    eps = rel_eps * nA
    ro = orc.randqb_b(A, eps, b, seed=3, omega_prec=8, storage_prec=16)
    Q, B, k, rc, st = _factor(rqb_lib, A, eps, b, 3)
    print("bf16 k", k, "oracle", ro.k, "D gpu", st.D[-2:], "D orc", ro.D[-2:], "eps2", eps * eps)
    assert rc == rqb_lib.RQB_OK
    _check_rank_d(k, ro, eps, b)
    assert orth_err(Q) <= 1e-5
    assert st.D[-1] <= eps * eps
    r = resid(A, Q, B)
    assert abs(r - np.sqrt(st.D[-1])) <= _stored_gap_bound(st.D, nA * nA)
    ro_gap = abs(resid(A, ro.Q, ro.B) - np.sqrt(ro.D[-1]))
    assert ro_gap <= _stored_gap_bound(ro.D, nA * nA)
    # at the GPU's rank (the oracle rerun to it in fixed-rank mode when a stop
    # decision fell inside the band): the per-block stored norms agree within
    # the roundings of the residual, and so do the residuals ||A - QB||_F
    rk = ro if k == ro.k else orc.randqb_b(A, 0.0, b, seed=3, max_rank=k, fixed_rank=True, omega_prec=8,
                                           storage_prec=16)
    nb = len(st.D)
    dg, do = np.sqrt(np.array(st.D)), np.sqrt(np.array(rk.D[:nb]))
    print("rel D gap", np.max(np.abs(dg - do) / do))
    assert np.all(np.abs(dg - do) <= 2.0 ** -9 * np.cumsum(do) + 1e-5 * nA)
    r_o = resid(A, rk.Q, rk.B)
    assert abs(r - r_o) <= (_stored_gap_bound(st.D, nA * nA) + _stored_gap_bound(rk.D, nA * nA)
                            + 2.0 ** -9 * np.sum(do) + 1e-5 * nA)


def test_randqb_fixed_rank_and_cap(orc, rqb_lib):
    m, n, b = 1800, 1100, 64
    A = _bf(orc, inputs.usv(m, n, inputs.spectrum_poly(min(m, n), 1.0), seed=4))
    ro = orc.randqb_b(A, 0.0, b, seed=8, max_rank=320, fixed_rank=True, omega_prec=8, storage_prec=16)
    Q, B, k, rc, st = _factor(rqb_lib, A, 0.0, b, 8, max_rank=320, fixed_rank=True)
    assert rc == rqb_lib.RQB_OK and k == 320 == ro.k
    assert orth_err(Q) <= 1e-5
    nA2 = float(np.sum(A * A))
    assert abs(resid(A, Q, B) - np.sqrt(st.D[-1])) <= _stored_gap_bound(st.D, nA2)
    assert abs(np.sqrt(st.D[-1]) - np.sqrt(ro.D[-1])) <= 2.0 ** -9 * np.sum(np.sqrt(ro.D)) + 1e-5 * np.sqrt(nA2)
    # the cap without fixed rank reports NOT_CONVERGED with valid factors
    Q, B, k, rc, _ = _factor(rqb_lib, A, 1e-9 * np.sqrt(nA2), b, 8, max_rank=192)
    assert rc == rqb_lib.RQB_NOT_CONVERGED and k == 192
    assert orth_err(Q) <= 1e-5


def test_bf16_unsupported_cases(rqb_lib):
    """Shapes below one TMA box and the power scheme are refused, not run elsewhere."""
    A = torch.zeros(100, 300, dtype=torch.bfloat16, device="cuda").t().contiguous().t()
    with rqb_lib.Handle(torch.bfloat16) as h:
        _, _, _, rc = h.rqb_factor(A, 1e-3, 32, 0, check=False)
        assert rc == rqb_lib.RQB_ERR_UNSUPPORTED
    with pytest.raises(rqb_lib.RqbError) as ei:
        rqb_lib.Handle(torch.bfloat16, power=1)
    assert ei.value.status == rqb_lib.RQB_ERR_UNSUPPORTED
    with pytest.raises(rqb_lib.RqbError):
        rqb_lib.Handle(torch.float32, prec=rqb_lib.RQB_PREC_BF16)


def test_randqb_nonfinite(orc, rqb_lib):
    A = np.ones((600, 400), dtype=np.float64)
    A[10, 20] = np.inf
    _, _, _, rc, _ = _factor(rqb_lib, A, 1e-3, 32, 0)
    assert rc == rqb_lib.RQB_ERR_NONFINITE


def test_randqb_bf16_vs_fp32_same_eps(orc, rqb_lib):
    """The BF16 handle and the plain FP32 handle on the same (BF16-exact)
    matrix and eps: ranks within a block, both residuals within eps plus the
    BF16 rounding gap."""
    m, n, b = 3000, 1600, 128
    A = _bf(orc, inputs.usv(m, n, inputs.spectrum_exp(min(m, n), 200), seed=12))
    eps = 1e-2 * np.linalg.norm(A)
    Qb, Bb, kb, rcb, st = _factor(rqb_lib, A, eps, b, 5)
    with rqb_lib.Handle(torch.float32) as h:
        Qn, Bn, kn, rcn = h.rqb_factor(to_dev(A, torch.float32), eps, b, 5, check=False)
        Qn, Bn = to_np(Qn), to_np(Bn)
    assert rcb == rcn == rqb_lib.RQB_OK
    assert abs(kb - kn) <= b
    assert resid(A, Qn, Bn) <= eps * (1 + 1e-4)
    assert resid(A, Qb, Bb) <= eps + _stored_gap_bound(st.D, float(np.sum(A * A)))


def test_randqb_zero_matrix(rqb_lib):
    Q, B, k, rc, st = _factor(rqb_lib, np.zeros((1000, 700)), 0.0, 128, 0)
    assert rc == rqb_lib.RQB_OK and k == 0


@pytest.mark.parametrize("m,n,p,col0", [(3000, 2000, 256, 128), (1037, 777, 37, 5), (129, 300, 64, 3)])
def test_omega_in_shared_memory_is_bitwise_the_buffered_sketch(orc, rqb_lib, m, n, p, col0):
    """RQB_FLAG_OMEGA_SMEM: Omega_i drawn by the sketch kernel into its
    shared-memory operand gives the same sketch as Omega_i from its buffer,
    bit for bit (same draws, same BF16 rounding, same MMA order), and so the
    same oracle parity (odd col0 exercises the unpaired Philox columns)."""
    rng = np.random.default_rng(m + n + p)
    A = _bf(orc, rng.standard_normal((m, n)))
    Ad = to_dev(A, torch.bfloat16)
    with rqb_lib.Handle(torch.bfloat16) as h0, rqb_lib.Handle(torch.bfloat16, flags=rqb_lib.RQB_FLAG_OMEGA_SMEM) as h1:
        Y0, n0 = h0.rqb_sketch(Ad, col0, p, seed=23)
        Y1, n1 = h1.rqb_sketch(Ad, col0, p, seed=23)
        Y0, Y1 = to_np(Y0), to_np(Y1)
        Om = to_np(h0.rqb_omega(n, col0, p, seed=23))
    assert np.array_equal(Y0, Y1) and n0 == n1
    # against the oracle entry by entry, with the few entries where the two
    # binary32 draws round to neighbouring BF16 values
    Yo = orc.sketch(A, 23, col0, p, omega_prec=8)
    Oo = orc.omega(23, n, col0, p, prec=8)
    assert_elementwise(Y1, Yo, product_bound(A, Oo), 1e-6, "BF16 sketch, Omega in shared memory",
                       extra=np.abs(A) @ np.abs(Om - Oo))


def test_omega_in_shared_memory_factorization_bitwise(orc, rqb_lib):
    m, n, b = 2049, 1300, 128
    A = _bf(orc, inputs.usv(m, n, inputs.spectrum_exp(min(m, n), 150), seed=31))
    eps = 1e-2 * np.linalg.norm(A)
    Q0, B0, k0, rc0, _ = _factor(rqb_lib, A, eps, b, 3)
    Q1, B1, k1, rc1, _ = _factor(rqb_lib, A, eps, b, 3, flags=rqb_lib.RQB_FLAG_OMEGA_SMEM)
    assert rc0 == rc1 == rqb_lib.RQB_OK and k0 == k1
    assert np.array_equal(Q0, Q1) and np.array_equal(B0, B1)


def test_omega_in_shared_memory_needs_bf16(rqb_lib):
    with pytest.raises(rqb_lib.RqbError) as ei:
        rqb_lib.Handle(torch.float32, flags=rqb_lib.RQB_FLAG_OMEGA_SMEM)
    assert ei.value.status == rqb_lib.RQB_ERR_UNSUPPORTED
