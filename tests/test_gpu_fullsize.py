"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (same recipes, seeds, handles and entry points):

  FP32 workload   20000 x 16000, s_j = j^-1.5, b = 128, eps = 1e-2 ||A||_F:
                  the whole factorization against the oracle (Fig. randQB_b,
                  binary32 Omega): rank exact, |r_gpu - r_orc| <= 1e-5 ||A||_F,
                  ||Q^T Q - I||_max <= 1e-5, and Q elementwise.
  batched         the 512-matrix batch factored in one rqb_factor_batched call;
                  a seeded subset of 16 matrices that includes the largest one
                  is compared with the oracle matrix by matrix (rank exact or one
                  block away inside the decision band, residual 1e-5 ||A_t||_F
                  at the GPU's rank, orthonormality 1e-5; a matrix factored to
                  its full rank min(m, n) is compared at k_prev, see
                  parity_util.assert_residual_parity).
  split-TF32 / BF16 workloads, 32768 x 16384, b = 256: the oracle cannot run
                  the whole factorization in seconds, so the first block is
                  compared with the oracle's (Q_1 = orth(A Omega_1) elementwise,
                  B_1 = Q_1^T A on sampled columns), and the whole run with what
                  holds at any size: ||Q^T Q - I||_max <= 1e-5, the residual
                  within eps and above the Eckart-Young tail (eq. minerrors),
                  k between the optimal eps-rank and two blocks above it, and the
                  residual the library reports equal to ||A - QB||_F computed
                  here in FP64.
Residuals and Gram matrices of the large factors are formed here with torch in
FP64 on the device (library products used as test instruments; the library
itself runs none of them).
"""
import numpy as np
import pytest
import torch

import inputs
from parity_util import (assert_elementwise, assert_residual_parity, check_rank, oracle_at_rank, orth_err,
                         product_bound, resid, to_np)

pytestmark = pytest.mark.gpu


def _dev_resid(A: torch.Tensor, Q: torch.Tensor, B: torch.Tensor) -> float:
    """||A - Q B||_F in FP64 on the device."""
    R = A.double()
    R -= Q.double() @ B.double()
    r = float(torch.linalg.norm(R))
    del R
    return r


def _dev_orth(Q: torch.Tensor) -> float:
    Qd = Q.double()
    G = Qd.T @ Qd
    G -= torch.eye(G.shape[0], dtype=torch.float64, device=G.device)
    return float(G.abs().max())


def _eps_rank(s: np.ndarray, eps: float) -> int:
    t = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])
    t = np.append(t, 0.0)
    return int(np.argmax(t <= eps))


def _tail(s: np.ndarray, k: int) -> float:
    return float(np.sqrt(np.sum(s[k:] ** 2)))


def test_fp32_workload_full_size_matches_oracle(orc, rqb_lib):
    A, meta = inputs.config_fp32_torch()          # bench's recipe and seed
    eps, b = meta["eps"], meta["b"]
    nA = meta["normA"]
    stream = torch.cuda.Stream()
    with rqb_lib.Handle(torch.float32, stream=stream, flags=rqb_lib.RQB_FLAG_PHASE_TIMING) as h:
        Q, B, k, rc = h.rqb_factor(A, eps, b, seed=0, check=False)
        torch.cuda.synchronize()
        r_g = _dev_resid(A, Q, B)
        o_g = _dev_orth(Q)
        Qn, Bn = to_np(Q), to_np(B)
    assert rc == rqb_lib.RQB_OK
    An = to_np(A)
    del A
    torch.cuda.empty_cache()
    ro = orc.randqb_b(An, eps, b, seed=0, omega_prec=32)
    r_o = resid(An, ro.Q, ro.B)
    print(f"FP32 full size: k {k} (oracle {ro.k}), residual {r_g / nA:.9e} (oracle {r_o / nA:.9e}), orth {o_g:.2e}")
    assert k == ro.k
    assert abs(r_g - r_o) <= 1e-5 * nA
    assert r_g <= eps * (1 + 1e-4)
    assert o_g <= 1e-5
    # diag(R) > 0 on both sides makes Q unique: an FP32 panel of kappa ~ 10^2
    # agrees with the FP64 one to a few 1e-6 relative
    assert np.abs(Qn - ro.Q).max() <= 1e-4
    assert np.abs(Bn - ro.B).max() <= 1e-4 * np.abs(ro.B).max()


def test_batched_workload_subset_matches_oracle(orc, rqb_lib):
    mats, eps, cases = inputs.config_batched_torch(512)   # bench's recipe and seeds
    b = 32
    sizes = np.array([c.m * c.n for c in cases])
    # the largest matrix (by m n) and the tallest one, then 14 drawn at random
    first = sorted({int(np.argmax(sizes)), int(np.argmax([c.m for c in cases]))})
    rng = np.random.default_rng(2024)
    rest = np.setdiff1d(np.arange(len(cases)), first)
    pick = first + [int(i) for i in rng.choice(rest, 16 - len(first), replace=False)]
    stream = torch.cuda.Stream()
    with rqb_lib.Handle(torch.float32, stream=stream) as h:
        out = h.rqb_factor_batched(mats, eps, b, seed=0)
        torch.cuda.synchronize()
        # the factors are views of the handle's buffers: read them before it closes
        got = {i: (to_np(out[i][0]), to_np(out[i][1]), out[i][2], out[i][3]) for i in pick}
    assert len(pick) == 16 and max(sizes[pick]) == sizes.max()
    for i in pick:
        A = to_np(mats[i])
        Q, B, k, st = got[i]
        nA = np.linalg.norm(A)
        ro = orc.randqb_b(A, eps[i], b, seed=0, omega_prec=32)
        print(f"batched {i}: {cases[i].m}x{cases[i].n} r={cases[i].rate} k {k} (oracle {ro.k})")
        assert st in (rqb_lib.RQB_OK, rqb_lib.RQB_NOT_CONVERGED), st
        assert st == (rqb_lib.RQB_OK if ro.status == 0 else rqb_lib.RQB_NOT_CONVERGED) or k != ro.k
        check_rank(k, ro, eps[i], b, rel_band=1e-3)
        rk = oracle_at_rank(orc, A, ro, k, b, 0, omega_prec=32)
        assert_residual_parity(A, Q, B, rk, 1e-5, b=b, eps=eps[i] if st == rqb_lib.RQB_OK else None)
        assert orth_err(Q) <= 1e-5


@pytest.mark.parametrize("form", ["tf32x3", "bf16"])
def test_tensor_core_workload_full_size(orc, rqb_lib, form):
    m, n, b = 32768, 16384, 256
    s = inputs.spectrum_mixed_config(min(m, n))
    nA = float(np.sqrt(np.sum(s ** 2)))
    A = inputs.usv_torch(m, n, s, 2, device="cuda", dtype=torch.float32)   # bench's recipe and seed
    if form == "bf16":
        Ab = torch.empty(n, m, dtype=torch.bfloat16, device="cuda").t()
        Ab.copy_(A)
        A = Ab
        eps, prec, oprec, dt = 1e-2 * nA, rqb_lib.RQB_PREC_BF16, 8, torch.bfloat16
    else:
        eps, prec, oprec, dt = 1e-3 * nA, rqb_lib.RQB_PREC_TF32X3, 19, torch.float32
    torch.cuda.empty_cache()
    stream = torch.cuda.Stream()
    with rqb_lib.Handle(dt, prec=prec, stream=stream, flags=rqb_lib.RQB_FLAG_PHASE_TIMING) as h:
        Q, B, k, rc = h.rqb_factor(A, eps, b, seed=0, check=False)
        torch.cuda.synchronize()
        st = h.rqb_get_stats()
        r_g = _dev_resid(A, Q, B)
        o_g = _dev_orth(Q)
        Q1 = to_np(Q[:, :b])
        J = np.sort(np.random.default_rng(5).choice(n, 48, replace=False))
        B1J = to_np(B[:b, :][:, torch.as_tensor(J, device="cuda")])
    An = to_np(A)
    nA_exact = float(np.linalg.norm(An))
    del A, Q, B
    torch.cuda.empty_cache()
    kopt = _eps_rank(s, eps)
    print(f"{form} full size: k {k} (optimal eps-rank {kopt}), residual {r_g / nA_exact:.6e}, orth {o_g:.2e}, "
          f"reported sqrt(D_s) {np.sqrt(st.D[-1]) / nA_exact:.6e}")
    assert rc == rqb_lib.RQB_OK
    assert o_g <= 1e-5
    if form == "tf32x3":
        # the matrix as stored (FP32) has the recipe's spectrum up to 1e-7
        # relative, far below eps
        assert r_g <= eps * (1 + 1e-4)
        assert r_g >= _tail(s, k) * (1 - 1e-4) - 1e-6 * nA
        assert kopt <= k <= (-(-kopt // b)) * b + 2 * b
        assert abs(r_g - np.sqrt(st.D[-1])) <= 4 * 2.0 ** -20 * (nA + np.sum(np.sqrt(st.D[:-1]))) + 1e-5 * nA
    else:
        # BF16 storage: the stored residual meets eps (line (6) on the stored
        # norm); A - QB differs from it by the roundings of the residual
        d = np.sqrt(np.asarray(st.D))
        gap = 1.01 * 2.0 ** -9 * d.sum() + 2e-5 * (nA_exact + d[:-1].sum())
        assert d[-1] <= eps
        assert abs(r_g - d[-1]) <= gap
        assert k >= kopt
    # the first block against the oracle's: Q_1 = orth(A Omega_1) (Fig. randQB_b
    # lines (2), (3)) and B_1 = Q_1^T A on sampled columns (line (4))
    Y1 = orc.sketch(An, 0, 0, b, omega_prec=oprec)
    Qo = orc.orth_reproject(Y1, None)
    del Y1
    dQ = Q1 - Qo
    dq = np.abs(dQ).max()
    AJ = An[:, J]
    Bo = Qo.T @ AJ
    print(f"{form} block 1: max |dQ| {dq:.2e}, max |dB| / max |B| {np.abs(B1J - Bo).max() / np.abs(Bo).max():.2e}")
    # Q_1: the sketch differs from the oracle's by the operand splits (2^-21 of
    # A for split-TF32; none for BF16, whose A is the BF16 input on both sides)
    # and FP32 sums; CholeskyQR2 of a well-conditioned panel keeps that level.
    assert dq <= 1e-4
    # B_1 = Q_1^T A from the GPU's own Q_1: B_gpu - Q_oracle^T A =
    # (Q_gpu - Q_oracle)^T A + the product's rounding, entry by entry
    assert_elementwise(B1J, Bo, product_bound(Qo.T, AJ), 4e-6 if form == "tf32x3" else 1e-5,
                       f"{form} B_1 = Q_1^T A", extra=np.abs(dQ).T @ np.abs(AJ))
