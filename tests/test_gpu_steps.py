"""Step-level parity of the CUDA path against the oracle (Fig. randQB_b lines (2)-(5)).

Each step runs through the C ABI on seeded inputs that span several tiles and
a ragged tail, and is compared element by element with the oracle's step:
  line (2)  Omega            FP64: within 5e-14 abs (libm vs CUDA transcendental ulps)
                             FP32: within 4 float ulps of the binary32 evaluation
  line (3)  A Omega, ||A||^2 FP64: 1e-12 relative (Frobenius), FP32: 1e-5
  line (3') orth + reproj.   FP64: 1e-10 elementwise; FP32: orthonormal to 1e-5
  line (4)  Q^T A, ||B||^2
  line (5)  A - Q B fused with the next A Omega
Beside each Frobenius check, every product entry is held to its own rounding
bound, |gpu - oracle|_ij <= rtol (|X| |Y|)_ij for X Y (plus, for the sketch,
|A| |Omega_gpu - Omega_oracle| from the generators' last-ulp differences):
rtol = 1e-14 for FP64 and 1e-6 for FP32 (about 16 u32: a partial sum of n
terms in FP32 drifts by ~u |x||y| per term on average).
"""
import numpy as np
import pytest
import torch

import inputs
from parity_util import assert_elementwise, orth_err, product_bound, to_dev, to_np

EL64, EL32 = 1e-14, 1e-6

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h64(rqb_lib):
    with rqb_lib.Handle(torch.float64) as h:
        yield h


@pytest.fixture(scope="module")
def h32(rqb_lib):
    with rqb_lib.Handle(torch.float32) as h:
        yield h


@pytest.mark.parametrize("n,col0,ncols", [(1000, 0, 50), (777, 7, 37), (3, 1, 5), (5000, 250, 128)])
def test_omega_fp64(orc, h64, n, col0, ncols):
    g = to_np(h64.rqb_omega(n, col0, ncols, seed=1234))
    o = orc.omega(1234, n, col0, ncols, prec=64)
    assert np.abs(g - o).max() <= 5e-14 * max(1.0, np.abs(o).max())


@pytest.mark.parametrize("n,col0,ncols", [(1000, 0, 64), (777, 3, 37), (4096, 256, 256)])
def test_omega_fp32(orc, h32, n, col0, ncols):
    g = to_np(h32.rqb_omega(n, col0, ncols, seed=99))
    o = orc.omega(99, n, col0, ncols, prec=32)
    assert np.all(np.abs(g - o) <= 4 * np.spacing(np.abs(o).astype(np.float32)).astype(np.float64) + 1e-7)


@pytest.mark.parametrize("m,n,p,col0", [(3000, 2000, 50, 0), (1037, 777, 37, 100), (130, 9, 5, 0), (2000, 1500, 128, 64)])
def test_sketch_fp64(orc, h64, m, n, p, col0):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    Y, nrm = h64.rqb_sketch(to_dev(A), col0, p, seed=7)
    Yo = orc.sketch(A, 7, col0, p, omega_prec=64)
    assert np.linalg.norm(to_np(Y) - Yo) <= 1e-12 * np.linalg.norm(Yo)
    assert abs(nrm - np.sum(A * A)) <= 1e-12 * np.sum(A * A)
    Om = orc.omega(7, n, col0, p, prec=64)
    dOm = 5e-14 * max(1.0, np.abs(Om).max())
    assert_elementwise(to_np(Y), Yo, product_bound(A, Om), EL64, "FP64 sketch",
                       extra=dOm * np.abs(A).sum(axis=1, keepdims=True))


@pytest.mark.parametrize("m,n,p", [(4000, 3000, 128), (1037, 777, 37), (2500, 1200, 256), (300, 4000, 32)])
def test_sketch_fp32(orc, h32, m, n, p):
    rng = np.random.default_rng(3 * m + n)
    A = rng.standard_normal((m, n)).astype(np.float32).astype(np.float64)
    Y, nrm = h32.rqb_sketch(to_dev(A, torch.float32), 0, p, seed=11)
    Yo = orc.sketch(A, 11, 0, p, omega_prec=32)
    assert np.linalg.norm(to_np(Y) - Yo) <= 1e-5 * np.linalg.norm(Yo)
    assert abs(nrm - np.sum(A * A)) <= 1e-9 * np.sum(A * A)
    Om = orc.omega(11, n, 0, p, prec=32)
    dOm = 4 * np.spacing(np.abs(Om).astype(np.float32)).astype(np.float64) + 1e-7
    assert_elementwise(to_np(Y), Yo, product_bound(A, Om), EL32, "FP32 sketch", extra=np.abs(A) @ dOm)


def test_sketch_padded_lda(orc, h64):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((301, 257))
    Y, _ = h64.rqb_sketch(to_dev(A, lda=333), 0, 20, seed=3)
    assert np.linalg.norm(to_np(Y) - orc.sketch(A, 3, 0, 20)) <= 1e-12 * np.linalg.norm(to_np(Y))


@pytest.mark.parametrize("m,p,kprev", [(2000, 50, 0), (2000, 50, 100), (1037, 37, 74), (700, 128, 256)])
def test_orth_fp64(orc, h64, m, p, kprev):
    rng = np.random.default_rng(m + p + kprev)
    Qbar = np.linalg.qr(rng.standard_normal((m, max(kprev, 1))))[0][:, :kprev]
    # a panel that is nearly orthogonal to Qbar, as A^(i-1) Omega is, with a spread spectrum
    Y = rng.standard_normal((m, p)) @ np.diag(np.logspace(0, -3, p))
    Y -= 1e-3 * Qbar @ (Qbar.T @ Y) if kprev else 0.0
    Qi = to_np(h64.rqb_orth(to_dev(Y), to_dev(Qbar) if kprev else None))
    Qo = orc.orth_reproject(Y, Qbar if kprev else None)
    assert np.abs(Qi - Qo).max() <= 1e-10
    assert orth_err(np.hstack([Qbar, Qi])) <= 1e-13


@pytest.mark.parametrize("m,p,kprev", [(4000, 128, 0), (4000, 128, 256), (1037, 37, 74), (3000, 256, 256)])
def test_orth_fp32(orc, h32, m, p, kprev):
    rng = np.random.default_rng(m + 2 * p + kprev)
    Qbar = np.linalg.qr(rng.standard_normal((m, max(kprev, 1))))[0][:, :kprev].astype(np.float32).astype(np.float64)
    Y = (rng.standard_normal((m, p)) @ np.diag(np.logspace(0, -2, p))).astype(np.float32).astype(np.float64)
    Qi = to_np(h32.rqb_orth(to_dev(Y, torch.float32), to_dev(Qbar, torch.float32) if kprev else None))
    Qo = orc.orth_reproject(Y, Qbar if kprev else None)
    assert orth_err(Qi) <= 1e-5
    if kprev:
        assert np.abs(Qbar.T @ Qi).max() <= 1e-5
    assert np.abs(Qi - Qo).max() <= 1e-3


@pytest.mark.parametrize("kind,cond,tol_q,route", [("f64", 1e1, 1e-10, 1), ("f64", 1e7, 1e-7, None),
                                                   ("f32", 1e1, 1e-4, 1), ("f32", 1e4, 1e-2, 1),
                                                   ("f32", 1e6, None, 0), ("tf32x3", 1e2, 1e-3, 1)])
@pytest.mark.parametrize("m,p", [(3000, 128), (2000, 256), (1500, 64)])
def test_orth_second_pass_routes(orc, rqb_lib, kind, cond, tol_q, route, m, p):
    """Lines (3), (3'): the second CholeskyQR pass takes its factor from the
    near-identity expansion when the first pass leaves ||E||_F = ||Y1^T Y1 -
    I||_F small (FP64 factor: first order below 2^-28; FP32 factor: first
    order below 1e-4, the iterated expansion below 2e-2) and from the
    elimination otherwise.  The FP32 handle's first pass leaves about
    u32 kappa(Y) there (its FP32 product Y R^-1), the split-TF32 one about
    1e-7 kappa(Y)^2: kappa = 10 takes first order, 1e4 on FP32 and 100 on
    split-TF32 the iteration, 1e6 on FP32 the elimination (1e7 in FP64 is
    near tau and may take either).  Both routes give an orthonormal Q_i equal
    to the oracle's, and stats.near_identity reports the route.  (FP64
    handles take blocks of up to 128 columns.)"""
    dtype = torch.float64 if kind == "f64" else torch.float32
    prec = rqb_lib.RQB_PREC_TF32X3 if kind == "tf32x3" else rqb_lib.RQB_PREC_NATIVE
    if dtype == torch.float64 and p > 128:
        p = 100
    rng = np.random.default_rng(int(m + p + np.log10(cond)))
    Y = np.linalg.qr(rng.standard_normal((m, p)))[0] @ np.diag(np.logspace(0, -np.log10(cond), p))
    Y = Y @ np.linalg.qr(rng.standard_normal((p, p)))[0]
    if dtype == torch.float32:
        Y = Y.astype(np.float32).astype(np.float64)
    with rqb_lib.Handle(dtype, prec=prec) as h:
        Qi = to_np(h.rqb_orth(to_dev(Y, dtype), None))
        st = h.rqb_get_stats()
    assert orth_err(Qi) <= (1e-13 if dtype == torch.float64 else 1e-5)
    if tol_q is not None:
        Qo = orc.orth_reproject(Y, None)
        assert np.abs(Qi - Qo).max() <= tol_q
    if route is not None and not (route == 0 and p < 128):
        # (a 64-column panel at kappa = 1e6 came out just inside the iterated
        # route's 2e-2: E grows with the panel width as well)
        assert st.near_identity == route


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
@pytest.mark.parametrize("m,n,p", [(3000, 2000, 50), (1037, 777, 37), (500, 4100, 128)])
def test_project(orc, rqb_lib, dtype, tol, m, n, p):
    rng = np.random.default_rng(m * n + p)
    A = rng.standard_normal((m, n))
    Q = np.linalg.qr(rng.standard_normal((m, p)))[0]
    if dtype == torch.float32:
        A = A.astype(np.float32).astype(np.float64)
        Q = Q.astype(np.float32).astype(np.float64)
    with rqb_lib.Handle(dtype) as h:
        Bi, nb2 = h.rqb_project(to_dev(Q, dtype), to_dev(A, dtype))
    Bo = Q.T @ A
    Bg = to_np(Bi)
    assert np.linalg.norm(Bg - Bo) <= tol * np.linalg.norm(Bo)
    assert abs(nb2 - np.sum(Bg * Bg)) <= 1e-12 * np.sum(Bg * Bg)
    assert_elementwise(Bg, Bo, product_bound(Q.T, A), EL64 if dtype == torch.float64 else EL32, "Q^T A")


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
@pytest.mark.parametrize("m,n,p,ncols,inplace", [(2000, 1000, 50, 50, False), (1037, 777, 37, 37, True),
                                                 (700, 2500, 128, 100, False), (300, 200, 64, 64, True)])
def test_downdate_sketch(orc, rqb_lib, dtype, tol, m, n, p, ncols, inplace):
    rng = np.random.default_rng(m + n + p + int(inplace))
    A = rng.standard_normal((m, n))
    Q = np.linalg.qr(rng.standard_normal((m, p)))[0]
    B = Q.T @ A
    prec = 64 if dtype == torch.float64 else 32
    if dtype == torch.float32:
        A, Q, B = (x.astype(np.float32).astype(np.float64) for x in (A, Q, B))
    Ad = to_dev(A, dtype)
    Wd = Ad if inplace else to_dev(np.zeros_like(A), dtype)
    with rqb_lib.Handle(dtype) as h:
        Y, nw2 = h.rqb_downdate_sketch(Ad, to_dev(Q, dtype), to_dev(B, dtype), Wd, 5 * p, ncols, seed=21)
    Wo = A - Q @ B
    Om = orc.omega(21, n, 5 * p, ncols, prec=prec)
    Yo = Wo @ Om
    assert np.linalg.norm(to_np(Wd) - Wo) <= tol * np.linalg.norm(A)
    assert np.linalg.norm(to_np(Y) - Yo) <= tol * np.linalg.norm(A) * np.sqrt(n)
    assert abs(nw2 - np.sum(Wo * Wo)) <= 10 * tol * np.sum(A * A)
    el = EL64 if dtype == torch.float64 else EL32
    wscale = np.abs(A) + product_bound(Q, B)
    assert_elementwise(to_np(Wd), Wo, wscale, el, "A - Q B")
    if dtype == torch.float64:
        dOm = 5e-14 * max(1.0, np.abs(Om).max()) * np.ones_like(Om)
    else:
        dOm = 4 * np.spacing(np.abs(Om).astype(np.float32)).astype(np.float64) + 1e-7
    assert_elementwise(to_np(Y), Yo, wscale @ np.abs(Om), el, "(A - Q B) Omega", extra=np.abs(Wo) @ dOm)
