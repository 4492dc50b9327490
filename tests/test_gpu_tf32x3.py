"""Split-TF32 tensor-core path (RQB_PREC_TF32X3) against the oracle.

The handle stores FP32 and runs the three products of Fig. randQB_b that read
all of A -- line (3) A Omega_i, line (4) Q_i^T A, line (5) A - Q_i B_i -- on
tcgen05 with hi/lo operand splits and FP32 accumulation; Omega_i is the
binary32 draw rounded to TF32, which the oracle reproduces with omega_prec=19.
A split operand keeps 2^-21 of each value, so the products carry FP32-level
error:
  steps      relative Frobenius error <= 2e-5 (as the FP32 SIMT steps)
  randQB_b   rank exact (or one block away when the oracle's stop quantity is
             within the rounding band of eps^2), ||Q^T Q - I||_max <= 1e-5,
             |r_gpu - r_oracle| <= 4 2^-20 sum_i ||A^(i)||_F + 1e-5 ||A||_F
Every step product is also checked entry by entry: |gpu - oracle|_ij <=
TOL_EL (|X| |Y|)_ij, TOL_EL = 4e-6 (a split product keeps 2^-21 of each term
and the FP32 sums of the tensor core round one way within a period), plus
|A| |Omega_gpu - Omega_oracle| for the sketch, whose TF32 draw differs from the
oracle's on a few entries by one TF32 ulp.
Shapes span several 128-row tiles, 32-column chunks and ragged tails; the
tensor-core path needs m >= 128 and n >= 256 (smaller shapes run the FP32
SIMT kernels, which one test checks).
"""
import numpy as np
import pytest
import torch

import inputs
from parity_util import (assert_elementwise, check_rank, oracle_at_rank, orth_err, product_bound, resid,
                         to_dev, to_np)

pytestmark = pytest.mark.gpu

TOL_STEP = 2e-5
TOL_EL = 4e-6


@pytest.fixture(scope="module")
def htc(rqb_lib):
    with rqb_lib.Handle(torch.float32, prec=rqb_lib.RQB_PREC_TF32X3) as h:
        yield h


def _f32(x):
    return x.astype(np.float32).astype(np.float64)


def test_omega_is_rounded_binary32_draw(orc, htc):
    g = to_np(htc.rqb_omega(3000, 40, 256, seed=99))
    o = orc.omega(99, 3000, 40, 256, prec=19)
    assert np.all(g == g.astype(np.float32).astype(np.float64))
    diff = g != o
    assert diff.mean() < 1e-3
    assert np.all(np.abs(g - o)[diff] <= 2.0 ** -10 * np.abs(o)[diff])


@pytest.mark.parametrize("m,n,p,col0", [(1000, 700, 64, 0), (3000, 2000, 256, 128), (1037, 777, 37, 5),
                                        (129, 257, 32, 0), (4100, 300, 128, 64)])
def test_sketch(orc, htc, m, n, p, col0):
    rng = np.random.default_rng(m + 3 * n + p)
    A = _f32(rng.standard_normal((m, n)))
    Y, nrm = htc.rqb_sketch(to_dev(A, torch.float32), col0, p, seed=17)
    Yo = orc.sketch(A, 17, col0, p, omega_prec=19)
    assert np.linalg.norm(to_np(Y) - Yo) <= TOL_STEP * np.linalg.norm(Yo)
    assert abs(nrm - np.sum(A * A)) <= 1e-9 * np.sum(A * A)
    Om = orc.omega(17, n, col0, p, prec=19)
    Omg = to_np(htc.rqb_omega(n, col0, p, seed=17))
    assert_elementwise(to_np(Y), Yo, product_bound(A, Om), TOL_EL, "split-TF32 sketch",
                       extra=np.abs(A) @ np.abs(Omg - Om))


def test_sketch_unaligned_lda(orc, htc):
    """lda not a multiple of 4: the matrix is copied to an aligned buffer first."""
    rng = np.random.default_rng(1)
    A = _f32(rng.standard_normal((1001, 600)))
    Y, _ = htc.rqb_sketch(to_dev(A, torch.float32, lda=1003), 0, 50, seed=2)
    Yo = orc.sketch(A, 2, 0, 50, omega_prec=19)
    assert np.linalg.norm(to_np(Y) - Yo) <= TOL_STEP * np.linalg.norm(Yo)


@pytest.mark.parametrize("m,n,p", [(3000, 2000, 50), (1037, 777, 37), (500, 4100, 128), (2048, 1024, 256)])
def test_project(orc, htc, m, n, p):
    rng = np.random.default_rng(m * n + p)
    A = _f32(rng.standard_normal((m, n)))
    Q = _f32(np.linalg.qr(rng.standard_normal((m, p)))[0])
    Bi, nb2 = htc.rqb_project(to_dev(Q, torch.float32), to_dev(A, torch.float32))
    Bo = Q.T @ A
    Bg = to_np(Bi)
    assert np.linalg.norm(Bg - Bo) <= TOL_STEP * np.linalg.norm(Bo)
    assert abs(nb2 - np.sum(Bg * Bg)) <= 1e-12 * np.sum(Bg * Bg)
    assert_elementwise(Bg, Bo, product_bound(Q.T, A), TOL_EL, "split-TF32 Q^T A")


@pytest.mark.parametrize("m,n,p,ncols,inplace", [(2000, 1000, 50, 50, False), (1037, 777, 37, 37, True),
                                                 (700, 2500, 128, 100, False), (300, 300, 64, 64, True),
                                                 (2500, 1300, 256, 256, False)])
def test_downdate_sketch(orc, htc, m, n, p, ncols, inplace):
    rng = np.random.default_rng(m + n + p + int(inplace))
    A = _f32(rng.standard_normal((m, n)))
    Q = _f32(np.linalg.qr(rng.standard_normal((m, p)))[0])
    B = _f32(Q.T @ A)
    Ad = to_dev(A, torch.float32)
    Wd = Ad if inplace else to_dev(np.zeros_like(A), torch.float32)
    Y, nw2 = htc.rqb_downdate_sketch(Ad, to_dev(Q, torch.float32), to_dev(B, torch.float32), Wd, 5 * p, ncols,
                                     seed=21)
    Wo = A - Q @ B
    Om = orc.omega(21, n, 5 * p, ncols, prec=19)
    Yo = Wo @ Om
    assert np.linalg.norm(to_np(Wd) - Wo) <= TOL_STEP * np.linalg.norm(A)
    assert np.linalg.norm(to_np(Y) - Yo) <= TOL_STEP * np.linalg.norm(A) * np.sqrt(n)
    assert abs(nw2 - np.sum(Wo * Wo)) <= 10 * TOL_STEP * np.sum(A * A)
    wscale = np.abs(A) + product_bound(Q, B)
    assert_elementwise(to_np(Wd), Wo, wscale, TOL_EL, "split-TF32 A - Q B")
    Omg = to_np(htc.rqb_omega(n, 5 * p, ncols, seed=21))
    assert_elementwise(to_np(Y), Yo, wscale @ np.abs(Om), TOL_EL, "split-TF32 (A - Q B) Omega",
                       extra=np.abs(Wo) @ np.abs(Omg - Om))


@pytest.mark.parametrize("m,p,kprev", [(4000, 128, 256), (3000, 256, 512), (1037, 37, 130), (4100, 64, 1000)])
def test_orth_tensor_core_reprojection(orc, htc, m, p, kprev):
    """kprev >= 128: line (3') runs on the tensor core (split-TF32 C = Qbar^T Y,
    C rounded to TF32 for Y -= Qbar C); the panel stays orthonormal and
    orthogonal to Qbar at the FP32 level and matches the oracle's Q_i."""
    rng = np.random.default_rng(m + 2 * p + kprev)
    Qbar = _f32(np.linalg.qr(rng.standard_normal((m, kprev)))[0])
    Y = rng.standard_normal((m, p)) @ np.diag(np.logspace(0, -2, p))
    Y = _f32(Y - (1 - 1e-3) * Qbar @ (Qbar.T @ Y))     # mostly, not exactly, orthogonal to Qbar
    Qi = to_np(htc.rqb_orth(to_dev(Y, torch.float32), to_dev(Qbar, torch.float32)))
    Qo = orc.orth_reproject(Y, Qbar)
    assert orth_err(Qi) <= 1e-5
    assert np.abs(Qbar.T @ Qi).max() <= 1e-5
    assert np.abs(Qi - Qo).max() <= 1e-3


@pytest.mark.parametrize("c2,fused", [(1e-6, 1), (0.04, 1), (0.07, 0), (30.0, 0)])
def test_orth_fused_second_gram(orc, htc, c2, fused):
    """Line (3') with kprev a multiple of 128: the second CholeskyQR pass takes
    its Gram from the product that gives C = Qbar^T Y1, as Y1^T Y1 - C^T C,
    where ||C||_F^2 <= 0.05, and from the re-projected panel otherwise.  Y is
    built so that its orthonormalised panel Y1 has ||C||_F^2 = c2 (Y1 =
    sqrt(1 - c^2) Z + c Qbar G, Z orthonormal and orthogonal to Qbar, G
    orthonormal, c^2 p = c2); both routes end orthonormal and equal to the
    oracle's Q_i, and stats.fused_gram reports the route.  Y -= Qbar C~ with
    C~ = C rounded to TF32 leaves Qbar^T Y = C - C~, at most 2^-11 |C| in each
    entry: Q_i is orthogonal to Qbar to 1e-5 plus twice that."""
    m, p, kprev = 3000, 256, 512
    rng = np.random.default_rng(int(1e3 * c2) + 5)
    X = np.linalg.qr(rng.standard_normal((m, kprev + p)))[0]
    Qbar, Z = X[:, :kprev], X[:, kprev:]
    G = np.linalg.qr(rng.standard_normal((kprev, p)))[0]
    c = np.sqrt(c2 / p)
    Y1 = np.sqrt(1 - c * c) * Z + c * (Qbar @ G)
    Y = _f32(Y1 @ np.diag(np.logspace(0, -1, p)) @ np.linalg.qr(rng.standard_normal((p, p)))[0])
    Qbar = _f32(Qbar)
    Qi = to_np(htc.rqb_orth(to_dev(Y, torch.float32), to_dev(Qbar, torch.float32)))
    st = htc.rqb_get_stats()
    Qo = orc.orth_reproject(Y, Qbar)
    cmax = np.abs(Qbar.T @ np.linalg.qr(Y)[0]).max()
    assert st.fused_gram == fused
    assert orth_err(Qi) <= 1e-5
    assert np.abs(Qbar.T @ Qi).max() <= 1e-5 + 2.0 ** -10 * cmax
    assert np.abs(Qi - Qo).max() <= 1e-3


@pytest.mark.parametrize("cond,fallback,fp32", [(1e1, 0, 1), (1e2, 0, 1), (1e3, 0, 0), (1e5, 1, 0)])
def test_orth_first_gram_fallback(orc, htc, cond, fallback, fp32):
    """The first CholeskyQR pass of a split-TF32 handle takes its Gram from the
    tensor core and factors it in FP32 when its pivots span at most 1e3
    (kappa(Y) = 10 and 100 here: spans 6.5 and 169), else in FP64 when they
    span at most 1e5 (kappa(Y) = 1e3: 1.0e4); kappa(Y) = 1e5 (span 3e7) is
    refactored from the exact FP64-accumulated Gram.  All end orthonormal and
    equal to the oracle's Q_i, and the stats report the route."""
    m, p = 6000, 256
    rng = np.random.default_rng(int(cond))
    U = np.linalg.qr(rng.standard_normal((m, p)))[0]
    V = np.linalg.qr(rng.standard_normal((p, p)))[0]
    Y = _f32((U * np.logspace(0, -np.log10(cond), p)) @ V.T)
    Qi = to_np(htc.rqb_orth(to_dev(Y, torch.float32), None))
    st = htc.rqb_get_stats()
    assert st.gram_fallbacks == fallback
    assert st.pass1_fp32 == fp32
    assert orth_err(Qi) <= 1e-5
    Qo = orc.orth_reproject(Y, None)
    assert np.abs(Qi - Qo).max() <= (1e-3 if cond < 1e3 else 5e-2)


def _factor(rqb, A, eps, b, seed, **kw):
    with rqb.Handle(torch.float32, prec=rqb.RQB_PREC_TF32X3, **kw) as h:
        Q, B, k, rc = h.rqb_factor(to_dev(A, torch.float32), eps, b, seed, check=False)
        st = h.rqb_get_stats()
        return to_np(Q), to_np(B), k, rc, st


def _resid_tol(ro, nA):
    S = nA + float(np.sum(np.sqrt(np.maximum(ro.D[:-1], 0.0))))
    return 4 * 2.0 ** -20 * S + 1e-5 * nA


@pytest.mark.parametrize("m,n,b,rate,rel_eps", [(1500, 1000, 64, 60, 1e-3), (2049, 1300, 128, 150, 1e-3),
                                                (1000, 1200, 50, 40, 1e-2), (4096, 2048, 256, 150, 1e-3),
                                                (700, 640, 32, 30, 5e-3)])
def test_randqb_matches_oracle(orc, rqb_lib, m, n, b, rate, rel_eps):
    s = inputs.spectrum_exp(min(m, n), rate)
    A = _f32(inputs.usv(m, n, s, seed=m + n))
    nA = np.linalg.norm(A)
    eps = rel_eps * nA
    ro = orc.randqb_b(A, eps, b, seed=3, omega_prec=19)
    Q, B, k, rc, st = _factor(rqb_lib, A, eps, b, 3)
    assert rc == rqb_lib.RQB_OK
    check_rank(k, ro, eps, b, rel_band=1e-3)
    assert orth_err(Q) <= 1e-5
    r = resid(A, Q, B)
    assert r <= eps * (1 + 1e-4)
    rk = oracle_at_rank(orc, A, ro, k, b, 3, omega_prec=19)
    assert abs(r - resid(A, rk.Q, rk.B)) <= _resid_tol(rk, nA)


def test_randqb_fixed_rank_and_cap(orc, rqb_lib):
    m, n, b = 1800, 1100, 64
    A = _f32(inputs.usv(m, n, inputs.spectrum_poly(min(m, n), 1.0), seed=4))
    ro = orc.randqb_b(A, 0.0, b, seed=8, max_rank=320, fixed_rank=True, omega_prec=19)
    Q, B, k, rc, _ = _factor(rqb_lib, A, 0.0, b, 8, max_rank=320, fixed_rank=True)
    assert rc == rqb_lib.RQB_OK and k == 320 == ro.k
    assert orth_err(Q) <= 1e-5
    assert abs(resid(A, Q, B) - resid(A, ro.Q, ro.B)) <= _resid_tol(ro, np.linalg.norm(A))
    # the cap without fixed rank reports NOT_CONVERGED with valid factors
    Q, B, k, rc, _ = _factor(rqb_lib, A, 1e-9 * np.linalg.norm(A), b, 8, max_rank=192)
    assert rc == rqb_lib.RQB_NOT_CONVERGED and k == 192
    assert orth_err(Q) <= 1e-5


def test_randqb_small_shape_runs_simt(orc, rqb_lib):
    """n < 256: the handle runs the FP32 SIMT products (binary32 Omega)."""
    m, n, b = 900, 200, 32
    A = _f32(inputs.usv(m, n, inputs.spectrum_exp(n, 20), seed=9))
    eps = 1e-3 * np.linalg.norm(A)
    ro = orc.randqb_b(A, eps, b, seed=1, omega_prec=32)
    Q, B, k, rc, _ = _factor(rqb_lib, A, eps, b, 1)
    assert rc == rqb_lib.RQB_OK
    check_rank(k, ro, eps, b, rel_band=1e-3)
    assert orth_err(Q) <= 1e-5
    rk = oracle_at_rank(orc, A, ro, k, b, 1, omega_prec=32)
    assert abs(resid(A, Q, B) - resid(A, rk.Q, rk.B)) <= 1e-5 * np.linalg.norm(A)


def test_randqb_nonfinite(rqb_lib):
    A = np.ones((600, 400), dtype=np.float64)
    A[10, 20] = np.nan
    _, _, _, rc, _ = _factor(rqb_lib, A, 1e-3, 32, 0)
    assert rc == rqb_lib.RQB_ERR_NONFINITE


def test_randqb_matches_native_fp32(rqb_lib):
    """Same matrix, same eps: the split-TF32 handle and the plain FP32 handle agree
    (rank within a block, residuals within the FP32 tolerance)."""
    m, n, b = 3000, 1600, 128
    A = _f32(inputs.usv(m, n, inputs.spectrum_exp(min(m, n), 200), seed=12))
    eps = 1e-3 * np.linalg.norm(A)
    Qt, Bt, kt, rct, _ = _factor(rqb_lib, A, eps, b, 5)
    with rqb_lib.Handle(torch.float32) as h:
        Qn, Bn, kn, rcn = h.rqb_factor(to_dev(A, torch.float32), eps, b, 5, check=False)
        Qn, Bn = to_np(Qn), to_np(Bn)
    assert rct == rcn == rqb_lib.RQB_OK
    assert abs(kt - kn) <= b
    assert resid(A, Qt, Bt) <= eps * (1 + 1e-4) and resid(A, Qn, Bn) <= eps * (1 + 1e-4)


def test_project_long_reduction_is_unbiased(htc):
    """K = m = 32768: each CTA reduces ~200 chunks.  The TMEM accumulator's
    one-sided rounding would shrink B by ~1e-4 over such a chain; the periodic
    drains keep the error at the split level and its mean below 1e-6."""
    m, n, p = 32768, 4096, 256
    rng = np.random.default_rng(77)
    A = rng.standard_normal((m, n), dtype=np.float32)
    Q = np.linalg.qr(rng.standard_normal((m, p)).astype(np.float32))[0].astype(np.float32)
    Bi, _ = htc.rqb_project(torch.from_numpy(Q).cuda().T.contiguous().T, torch.from_numpy(A).cuda().T.contiguous().T)
    J = rng.choice(n, 96, replace=False)
    Bo = Q.astype(np.float64).T @ A[:, J].astype(np.float64)
    Bg = to_np(Bi)[:, J]
    print("project rel", np.linalg.norm(Bg - Bo) / np.linalg.norm(Bo), "bias", np.sum((Bg - Bo) * Bo) / np.sum(Bo * Bo))
    assert np.linalg.norm(Bg - Bo) <= 2e-6 * np.linalg.norm(Bo)
    assert abs(np.sum((Bg - Bo) * Bo)) <= 1e-6 * np.sum(Bo * Bo)     # no systematic shrink


def test_sketch_long_reduction_is_unbiased(orc, htc):
    """K = n = 32768.  The product is checked against the handle's own Omega
    (rqb_omega), which equals the oracle's TF32 draw except where the binary32
    Box-Muller of CUDA and of libm (about 1 ulp apart) round to different TF32
    neighbours."""
    m, n, p = 4096, 32768, 256
    rng = np.random.default_rng(78)
    A = rng.standard_normal((m, n), dtype=np.float32)
    Y, _ = htc.rqb_sketch(torch.from_numpy(A).cuda().T.contiguous().T, 0, p, seed=5)
    Om = to_np(htc.rqb_omega(n, 0, p, seed=5))
    Oo = orc.omega(5, n, 0, p, prec=19)
    diff = Om != Oo
    assert diff.mean() < 1e-3
    assert np.all(np.abs(Om - Oo)[diff] <= 2.0 ** -10 * np.abs(Oo)[diff])
    I = rng.choice(m, 64, replace=False)
    Yo = A[I].astype(np.float64) @ Om
    Yg = to_np(Y)[I]
    print("sketch rel", np.linalg.norm(Yg - Yo) / np.linalg.norm(Yo), "bias", np.sum((Yg - Yo) * Yo) / np.sum(Yo * Yo),
          "omega mismatch", diff.mean())
    assert np.linalg.norm(Yg - Yo) <= 2e-6 * np.linalg.norm(Yo)
    assert abs(np.sum((Yg - Yo) * Yo)) <= 1e-6 * np.sum(Yo * Yo)


def test_bounded_wait_times_out_and_context_survives(rqb_lib):
    """The failure path of the tensor-core kernels: a wait on an mbarrier that
    nothing completes gives up after its 2 s limit with RQB_ERR_TIMEOUT, and the
    same handle then factors normally."""
    with rqb_lib.Handle(torch.float32, prec=rqb_lib.RQB_PREC_TF32X3) as h:
        rc, ms = h.rqb_wait_selftest()
        assert rc == rqb_lib.RQB_ERR_TIMEOUT
        assert 1500.0 <= ms <= 4000.0
        A = torch.randn(600, 400, device="cuda").t().contiguous().t()
        _, _, k, rc = h.rqb_factor(A, 0.5 * float(A.norm()), 32, 0)
        assert rc == rqb_lib.RQB_OK and k > 0


def test_randqb_zero_matrix(rqb_lib):
    """A = 0: the empty factorization (k = 0, RQB_OK), not a breakdown of the
    zero sketch."""
    Q, B, k, rc, st = _factor(rqb_lib, np.zeros((1000, 700)), 0.0, 128, 0)
    assert rc == rqb_lib.RQB_OK and k == 0
