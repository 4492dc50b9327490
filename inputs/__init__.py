"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the factorization's arithmetic: it only builds test
matrices with prescribed singular values, the way the paper builds its test
matrices (Sec. 6.2: A = U D V^* with U, V the orthonormal factors of a QR of a
random Gaussian matrix), and the workload recipes of the benchmark.  The
Gaussian test matrix Omega is not an input: both the oracle and the GPU path
draw it from the seed.

Recipes (sizes and spectra):
  config_fp64      2000 x 1000, s_j = 10^(-8 (j-1)/999), b = 50, eps = 1e-4 ||A||_F
  config_fp32      20000 x 16000, s_j = j^-1.5, b = 128, eps = 1e-2 ||A||_F
  config_mixed     32768 x 16384, s_j = 10^(-4 j/2000) for j <= 2000, then 1e-6,
                   b = 256, eps = 1e-3 ||A||_F
  config_batched   512 matrices, m ~ U[256, 4096], n ~ U[128, min(m, 2048)],
                   s_j = exp(-j/r), r ~ U[10, 200], b = 32, eps_t = 1e-3 ||A_t||_F
                   (config_batched_torch builds the whole batch on the device)
  config_adjoint   8192 x 4096, N(0,1)/sqrt(4096) + planted rank 64 of norm 10,
                   k = 256 fixed, b = 64
  matrix1/2/4      the paper's Matrices 1, 2 and 4 (Sec. 6.2)
U and V are the Q factors (sign-normalised, diag(R) > 0) of the QR of seeded
iid N(0,1) matrices.  Small cases are built with numpy in FP64; the large ones
are built with torch on the current device (a library QR and GEMM) and
returned as FP32 device tensors.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------------
# spectra
def spectrum_fp64_config(n: int = 1000) -> np.ndarray:
    j = np.arange(1, n + 1, dtype=np.float64)
    return 10.0 ** (-8.0 * (j - 1) / (n - 1))


def spectrum_poly(r: int, power: float = 1.5) -> np.ndarray:
    j = np.arange(1, r + 1, dtype=np.float64)
    return j ** (-power)


def spectrum_mixed_config(r: int, knee: int = 2000, tail: float = 1e-6) -> np.ndarray:
    j = np.arange(1, r + 1, dtype=np.float64)
    s = 10.0 ** (-4.0 * j / knee)
    s[j > knee] = tail
    return s


def spectrum_exp(r: int, rate: float) -> np.ndarray:
    j = np.arange(1, r + 1, dtype=np.float64)
    return np.exp(-j / rate)


# --------------------------------------------------------------------------
# numpy (FP64) builders
def haar_factor(rows: int, cols: int, rng: np.random.Generator) -> np.ndarray:
    """Q factor of the Householder QR of an iid N(0,1) rows x cols matrix, diag(R) > 0."""
    G = rng.standard_normal((rows, cols))
    Qf, R = np.linalg.qr(G, mode="reduced")
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return np.asfortranarray(Qf * sgn)


def usv(m: int, n: int, s: np.ndarray, seed: int) -> np.ndarray:
    """A = U diag(s) V^T, U m x r, V n x r, r = len(s) <= min(m, n)."""
    r = len(s)
    rng = np.random.default_rng(seed)
    U = haar_factor(m, r, rng)
    V = haar_factor(n, r, rng)
    return np.asfortranarray((U * s) @ V.T)


def config_fp64(seed: int = 1) -> tuple[np.ndarray, dict]:
    m, n = 2000, 1000
    s = spectrum_fp64_config(n)
    A = usv(m, n, s, seed)
    nrm = float(np.sqrt(np.sum(s ** 2)))
    return A, dict(m=m, n=n, b=50, eps=1e-4 * nrm, seed_omega=0, sigma=s, normA=nrm)


def matrix1(m: int = 800, n: int = 600, seed: int = 11, beta: float = 0.65) -> tuple[np.ndarray, np.ndarray]:
    """Matrix 1 of Sec. 6.2: d_j = g_j^2 beta^(j-1), g_j ~ U[0, 1]."""
    rng = np.random.default_rng(seed)
    r = min(m, n)
    g = rng.uniform(0.0, 1.0, size=r)
    d = g ** 2 * beta ** np.arange(r)
    U = haar_factor(m, r, rng)
    V = haar_factor(n, r, rng)
    return np.asfortranarray((U * d) @ V.T), d


def matrix2(m: int = 800, n: int = 600, seed: int = 12) -> tuple[np.ndarray, np.ndarray]:
    """Matrix 2 of Sec. 6.2, read with a decaying exponent: d_j = (1 + 200 (j-1))^(-1/2)."""
    rng = np.random.default_rng(seed)
    r = min(m, n)
    d = (1.0 + 200.0 * np.arange(r)) ** -0.5
    U = haar_factor(m, r, rng)
    V = haar_factor(n, r, rng)
    return np.asfortranarray((U * d) @ V.T), d


def matrix4(n: int = 1000, seed: int = 14) -> np.ndarray:
    """Matrix 4 of Sec. 6.2 (Kahan variant): S K with S = diag(zeta^(j-1)),
    K unit upper triangular with -phi above the diagonal, zeta^2 + phi^2 = 1."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.05, 0.5)
    zeta = math.sqrt(1.0 - phi * phi)
    S = zeta ** np.arange(n)
    K = np.triu(-phi * np.ones((n, n)), 1) + np.eye(n)
    return np.asfortranarray(S[:, None] * K)


# --------------------------------------------------------------------------
# batched recipe
@dataclass
class BatchedCase:
    m: int
    n: int
    rate: int          # r of s_j = exp(-j / r)


def batched_sizes(count: int = 512, seed: int = 0, m_lo: int = 256, m_hi: int = 4096,
                  n_lo: int = 128, n_hi: int = 2048, r_lo: int = 10, r_hi: int = 200) -> list[BatchedCase]:
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(m_lo, m_hi + 1))
        n = int(rng.integers(n_lo, min(m, n_hi) + 1))
        r = int(rng.integers(r_lo, r_hi + 1))
        out.append(BatchedCase(m, n, r))
    return out


def batched_matrix_np(case: BatchedCase, seed: int) -> np.ndarray:
    r = min(case.m, case.n)
    return usv(case.m, case.n, spectrum_exp(r, case.rate), seed)


# --------------------------------------------------------------------------
# torch builders for the large workloads (device-side library QR / GEMM)
def _torch():
    import torch
    return torch


def _preload_torch_linalg(torch):
    """torch loads its CUDA linear-algebra library lazily by soname; under a
    profiler's injection that lookup can fail, so load it by path first."""
    import ctypes
    import os
    path = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(path):
        try:
            ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
        except OSError:
            pass


def usv_torch(m: int, n: int, s: np.ndarray, seed: int, device="cuda", dtype=None):
    """A = U diag(s) V^T built with torch on `device`; QR and GEMM run in FP32
    with TF32 disabled (FP64 when dtype is float64).  Returns an (m, n) tensor
    whose storage is column-major (a transposed view of a contiguous n x m)."""
    torch = _torch()
    _preload_torch_linalg(torch)
    dtype = dtype or torch.float32
    r = len(s)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    prev = torch.backends.cuda.matmul.allow_tf32 if str(device).startswith("cuda") else None
    if prev is not None:
        torch.backends.cuda.matmul.allow_tf32 = False
    try:
        def haar(rows, cols):
            G = torch.randn(rows, cols, generator=g, device=device, dtype=dtype)
            Qf, R = torch.linalg.qr(G, mode="reduced")
            sg = torch.sign(torch.diagonal(R))
            sg[sg == 0] = 1
            return Qf * sg
        U = haar(m, r)
        V = haar(n, r)
        sv = torch.as_tensor(s, device=device, dtype=dtype)
        At = (V * sv) @ U.T          # n x m row-major == A column-major
        del U, V
    finally:
        if prev is not None:
            torch.backends.cuda.matmul.allow_tf32 = prev
    return At.T                      # m x n view, column-major storage


def config_fp32_torch(m: int = 20000, n: int = 16000, seed: int = 2, device="cuda"):
    s = spectrum_poly(min(m, n))
    nrm = float(np.sqrt(np.sum(s ** 2)))
    A = usv_torch(m, n, s, seed, device=device)
    return A, dict(m=m, n=n, b=128, eps=1e-2 * nrm, seed_omega=0, sigma=s, normA=nrm)


def config_mixed_torch(m: int = 32768, n: int = 16384, seed: int = 3, device="cuda", knee: int = 2000):
    s = spectrum_mixed_config(min(m, n), knee=knee)
    nrm = float(np.sqrt(np.sum(s ** 2)))
    A = usv_torch(m, n, s, seed, device=device)
    return A, dict(m=m, n=n, b=256, eps=1e-3 * nrm, seed_omega=0, sigma=s, normA=nrm)


def config_batched_torch(count: int = 512, seed: int = 0, device="cuda"):
    """The batched workload on `device`: sizes and rates from batched_sizes
    (seed), matrix t built by usv_torch with seed 1000 + t, eps_t = 1e-3
    ||A_t||_F (from the spectrum).  Returns (matrices, eps list, cases)."""
    torch = _torch()
    cases = batched_sizes(count, seed=seed)
    mats, eps = [], []
    for i, c in enumerate(cases):
        s = spectrum_exp(min(c.m, c.n), c.rate)
        mats.append(usv_torch(c.m, c.n, s, 1000 + i, device=device, dtype=torch.float32))
        eps.append(1e-3 * float(np.sqrt(np.sum(s ** 2))))
    return mats, eps, cases


def config_adjoint_np(m: int = 8192, n: int = 4096, seed: int = 5, rank: int = 64, norm: float = 10.0):
    rng = np.random.default_rng(seed)
    N = rng.standard_normal((m, n)) / math.sqrt(n)
    U = haar_factor(m, rank, rng)
    V = haar_factor(n, rank, rng)
    sig = np.full(rank, norm / math.sqrt(rank))
    A = np.asfortranarray(N + (U * sig) @ V.T)
    T = np.asfortranarray(rng.standard_normal((m, n)))
    return A, T, dict(m=m, n=n, b=64, k=256)
