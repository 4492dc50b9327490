"""Pins of the oracle's single-step functions, which the GPU step tests use as
their truth, against what the mathematics fixes independently of the oracle:

  orc_sketch (Fig. randQB_b line (3), Y = A Omega_i with Omega_i the global
  columns col0 .. col0 + p - 1 of one Gaussian matrix, eq. OmegaBlock):
    * A = I gives Omega_i itself, bit for bit, and a row-selection matrix gives
      the selected rows of Omega_i: every index (row, global column, col0 and
      the strides of A and Y) shows up in an exact result;
    * slicing: the sketch with col0 = c equals columns c .. of the sketch with
      col0 = 0 (eq. OmegaBlock), bit for bit;
    * a dense A agrees with the plain product A @ Omega to rounding.

  orc_orth_reproject (lines (3), (3'): Q_i = orth(Y), Q_i = orth(Q_i - Qbar Qbar^T Q_i)):
    in exact arithmetic the result is the Q factor, with positive diagonal, of
    the projected panel (I - Qbar Qbar^T) Y: Y = Q1 R1 and
    (I - Qbar Qbar^T) Q1 = Q_i R2 give (I - Qbar Qbar^T) Y = Q_i (R2 R1) with R2 R1
    upper triangular and positive on its diagonal, and that factor is unique for
    a full-rank panel (Sec. 2.4 with the diag(R) > 0 convention).  So:
    * Q_i matches LAPACK's QR of (I - Qbar Qbar^T) Y, sign-fixed;
    * Q_i is orthonormal and orthogonal to Qbar;
    * T = Q_i^T (I - Qbar Qbar^T) Y is upper triangular with a positive diagonal
      and reproduces the projected panel (Gram-Schmidt column order kept);
    * kprev = 0 reduces to orth(Y).
"""
import numpy as np
import pytest


def _lapack_q(Y):
    Qn, Rn = np.linalg.qr(Y, mode="reduced")
    s = np.sign(np.diag(Rn))
    s[s == 0] = 1
    return Qn * s


def _orthonormal(m, k, seed):
    return _lapack_q(np.random.default_rng(seed).standard_normal((m, k)))


# --------------------------------------------------------------------------- sketch

@pytest.mark.parametrize("n,col0,p,prec", [(40, 0, 8, 64), (37, 5, 11, 64), (64, 130, 32, 32),
                                           (33, 7, 3, 19), (50, 9, 16, 8)])
@pytest.mark.parametrize("pads", [(0, 0), (3, 5)])
def test_sketch_of_identity_is_omega(orc, n, col0, p, prec, pads):
    A = np.eye(n)
    Y = orc.sketch(A, seed=11, col0=col0, p=p, omega_prec=prec, lda_pad=pads[0], ldy_pad=pads[1])
    Om = orc.omega(11, n, col0, p, prec=prec)
    assert np.array_equal(Y, Om)


@pytest.mark.parametrize("pads", [(0, 0), (2, 7)])
def test_sketch_of_row_selection_picks_omega_rows(orc, pads):
    n, m, col0, p = 29, 13, 6, 9
    rng = np.random.default_rng(4)
    rows = rng.choice(n, size=m, replace=True)
    A = np.zeros((m, n))
    A[np.arange(m), rows] = 1.0
    Y = orc.sketch(A, seed=3, col0=col0, p=p, lda_pad=pads[0], ldy_pad=pads[1])
    Om = orc.omega(3, n, col0, p)
    assert np.array_equal(Y, Om[rows, :])
    # scaling a selection by a power of two scales the rows exactly
    Y2 = orc.sketch(4.0 * A, seed=3, col0=col0, p=p)
    assert np.array_equal(Y2, 4.0 * Om[rows, :])


def test_sketch_slices_one_omega(orc):
    rng = np.random.default_rng(7)
    A = rng.standard_normal((45, 31))
    full = orc.sketch(A, seed=5, col0=0, p=24)
    for c, p in [(0, 8), (8, 8), (16, 8), (3, 13), (23, 1)]:
        part = orc.sketch(A, seed=5, col0=c, p=p)
        assert np.array_equal(part, full[:, c:c + p])


@pytest.mark.parametrize("m,n,col0,p", [(60, 45, 0, 10), (33, 70, 21, 7), (128, 128, 256, 32)])
def test_sketch_dense_matches_product(orc, m, n, col0, p):
    rng = np.random.default_rng(m + n + p)
    A = rng.standard_normal((m, n))
    Y = orc.sketch(A, seed=2, col0=col0, p=p, lda_pad=1, ldy_pad=4)
    Om = orc.omega(2, n, col0, p)
    ref = A @ Om
    assert np.abs(Y - ref).max() <= 1e-13 * np.abs(A).sum(axis=1).max() * np.abs(Om).max()
    # a different seed or a shifted col0 gives a different sketch
    assert np.abs(orc.sketch(A, seed=3, col0=col0, p=p) - Y).max() > 1e-3
    assert np.abs(orc.sketch(A, seed=2, col0=col0 + 1, p=p) - Y).max() > 1e-3


# ------------------------------------------------------------------- orth + (3')

@pytest.mark.parametrize("m,kprev,p", [(200, 0, 16), (200, 24, 16), (300, 100, 40), (97, 50, 7),
                                       (64, 48, 16)])
@pytest.mark.parametrize("ld_pad", [0, 5])
@pytest.mark.parametrize("inside", [False, True])
def test_orth_reproject_is_qr_of_projected_panel(orc, m, kprev, p, ld_pad, inside):
    rng = np.random.default_rng(m * 7 + kprev + p)
    Qbar = _orthonormal(m, kprev, seed=m + kprev) if kprev else np.zeros((m, 0))
    # columns of very different scale; with inside=True also a large component
    # inside span(Qbar), as in a panel sketched from a residual with rounding
    Y = rng.standard_normal((m, p)) @ np.diag(np.logspace(0, -3, p))
    if kprev and inside:
        Y = Y + Qbar @ rng.standard_normal((kprev, p))
    Qi = orc.orth_reproject(Y, Qbar, ld_pad=ld_pad)
    Yp = Y - Qbar @ (Qbar.T @ Y)

    assert np.abs(Qi.T @ Qi - np.eye(p)).max() < 1e-13
    if kprev:
        # one projection leaves about u ||Y|| / sigma_min((I - Qbar Qbar^T) Y)
        # of Qbar in Q_i; a panel with little of Qbar in it is orthogonal to it
        # to a few u
        sv = np.linalg.svd(Yp, compute_uv=False)
        grow = np.linalg.norm(Y, 2) / sv[-1]
        bound = 1e-13 if not inside else 64 * 2.0 ** -52 * grow
        assert np.abs(Qbar.T @ Qi).max() < bound
    T = Qi.T @ Yp
    scale = np.linalg.norm(Yp, axis=0)
    assert np.all(np.abs(np.tril(T, -1)) <= 1e-12 * scale[None, :])
    assert np.all(np.diag(T) > 0)
    assert np.abs(Qi @ T - Yp).max() <= 1e-12 * scale.max()
    ref = _lapack_q(Yp)
    assert np.abs(Qi - ref).max() < 1e-9


def test_orth_reproject_without_qbar_is_orth(orc):
    rng = np.random.default_rng(12)
    Y = rng.standard_normal((150, 20))
    Qi = orc.orth_reproject(Y, None)
    assert np.abs(Qi - orc.orth(Y)).max() < 1e-13
    assert np.abs(Qi - _lapack_q(Y)).max() < 1e-12


def test_orth_reproject_drops_the_qbar_component(orc):
    """Y = Qbar X + Z with Z orthogonal to Qbar: the result depends on Z only."""
    m, kprev, p = 120, 30, 12
    rng = np.random.default_rng(21)
    Qbar = _orthonormal(m, kprev, seed=5)
    Z = rng.standard_normal((m, p))
    Z -= Qbar @ (Qbar.T @ Z)
    X = 1e3 * rng.standard_normal((kprev, p))
    Qa = orc.orth_reproject(Qbar @ X + Z, Qbar)
    Qz = orc.orth_reproject(Z, Qbar)
    # the (3) orth of a panel dominated by Qbar X loses about kappa u of Z's
    # direction; line (3') recovers the rest
    assert np.abs(Qa - Qz).max() < 1e-9
    assert np.abs(Qz - _lapack_q(Z)).max() < 1e-12
