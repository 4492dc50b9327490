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
