"""Helpers shared by the GPU parity tests (conversions, tolerances, rank ties)."""
import numpy as np
import torch


def to_dev(A: np.ndarray, dtype=torch.float64, lda: int | None = None) -> torch.Tensor:
    """Column-major device copy of A (optionally inside a taller buffer, leading dim lda)."""
    m, n = A.shape
    ld = lda or m
    buf = torch.zeros(n, ld, dtype=dtype, device="cuda")
    buf[:, :m] = torch.as_tensor(np.ascontiguousarray(A.T), dtype=dtype, device="cuda")
    return buf.t()[:m, :]


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().to("cpu", torch.float64).numpy()


def orth_err(Q: np.ndarray) -> float:
    return float(np.abs(Q.T @ Q - np.eye(Q.shape[1])).max()) if Q.shape[1] else 0.0


def resid(A: np.ndarray, Q: np.ndarray, B: np.ndarray) -> float:
    return float(np.linalg.norm(A - Q @ B))


def rank_tie(orc_res, eps: float, rel_band: float) -> bool:
    """True when the oracle's stop decision is within rel_band of eps^2 at the
    last or second-to-last block, so that a GPU rank one block away is also valid."""
    e2 = eps * eps
    Es = list(orc_res.E)
    cands = [Es[-1]] + ([Es[-2]] if len(Es) > 1 else [])
    return any(abs(E - e2) <= rel_band * e2 for E in cands)


def check_rank(k_gpu: int, orc_res, eps: float, b: int, rel_band: float):
    if k_gpu == orc_res.k:
        return
    assert rank_tie(orc_res, eps, rel_band) and abs(k_gpu - orc_res.k) <= b, \
        f"rank {k_gpu} != oracle {orc_res.k} (E tail {orc_res.E[-2:]}, eps^2 {eps * eps})"


def oracle_at_rank(orc, A: np.ndarray, orc_res, k_gpu: int, b: int, seed: int, **kw):
    """The oracle's factorization at the GPU's rank.  When the GPU stopped one
    block earlier or later than the oracle (a stop quantity inside the rounding
    band of eps^2), the oracle is rerun in fixed-rank mode to k_gpu: the same
    Omega gives the same first blocks, so its residual at k_gpu is the one the
    GPU's must match.  kw: the oracle's precision modes (omega_prec, ...)."""
    if k_gpu == orc_res.k:
        return orc_res
    return orc.randqb_b(A, 0.0, b, seed=seed, max_rank=k_gpu, fixed_rank=True, **kw)


def product_bound(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """(|X| |Y|)_ij: the scale of the rounding error of entry (i, j) of X Y
    computed in floating point (sum_k |x_ik| |y_kj| times a small multiple of
    the unit roundoff)."""
    return np.abs(X) @ np.abs(Y)


def assert_elementwise(G: np.ndarray, O: np.ndarray, bound: np.ndarray, rtol: float, what: str = "",
                       extra: np.ndarray | float = 0.0):
    """|G - O| <= rtol * bound + extra entry by entry.  A Frobenius check lets
    an error confined to one tile or a ragged edge hide behind the rest of the
    matrix; this one does not."""
    assert G.shape == O.shape, (G.shape, O.shape)
    err = np.abs(G - O)
    lim = rtol * bound + extra
    bad = err > lim
    if bad.any():
        idx = np.unravel_index(np.argmax(err / np.maximum(lim, 1e-300)), err.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} of {err.size} entries beyond the elementwise bound; "
                             f"worst at {idx}: |diff| {err[idx]:.3e} > {lim[idx] if np.ndim(lim) else lim:.3e}")


def assert_residual_parity(A: np.ndarray, Q: np.ndarray, B: np.ndarray, ro, tol: float, b: int | None = None,
                           eps: float | None = None, fp32_cap: bool = True):
    """|r_gpu - r_orc| <= tol ||A||_F with r = ||A - QB||_F from each side's
    factors, ro the oracle at the GPU's rank.

    The rank cap is the one exception (fp32_cap): when the last block is
    shrunk to the p = min(m, n) - k_prev columns left, its sketch has no
    oversampling, so the subspace it finds moves with the rounding of the
    stored residual by about u ||A^(i)|| / sigma_min(A^(s-1) Omega_s), which
    in FP32 can exceed tol ||A||.  There the residuals are compared at k_prev
    (all blocks but the last, to tol), and the last block is held to what it
    must do in any precision: not raise the residual, and meet eps when the
    run stopped on it."""
    nA = float(np.linalg.norm(A))
    m, n = A.shape
    k = Q.shape[1]
    r_g, r_o = resid(A, Q, B), resid(A, ro.Q, ro.B)
    if abs(r_g - r_o) <= tol * nA:
        return
    cap = min(m, n)
    if not (fp32_cap and k == ro.k == cap and ro.blocks > 1):
        raise AssertionError(f"residual {r_g / nA:.3e} vs oracle {r_o / nA:.3e} (tol {tol})")
    if b is None:
        raise AssertionError("rank cap: pass the block size b")
    kprev = b * (ro.blocks - 1)
    rg_prev = resid(A, Q[:, :kprev], B[:kprev])
    ro_prev = resid(A, ro.Q[:, :kprev], ro.B[:kprev])
    assert abs(rg_prev - ro_prev) <= tol * nA, \
        f"rank cap: residual at k_prev={kprev} {rg_prev / nA:.3e} vs oracle {ro_prev / nA:.3e}"
    assert r_g <= rg_prev * (1 + 1e-6) + tol * nA, "rank cap: the last block raised the residual"
    if eps is not None:
        assert r_g <= eps * (1 + 1e-4), "rank cap: the run stopped with a residual above eps"
