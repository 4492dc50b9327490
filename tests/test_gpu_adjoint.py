"""rqb_backward: gradient through the fixed-rank map X = Q Q^T A (Omega held fixed).

The gradient depends on A, Omega and G only (Q Q^T is the projector onto
R(A Omega)), not on the basis Q, so the GPU gradient (from the GPU's Q, B) is
compared with the oracle's (from the oracle's Q, B):
  FP64  relative Frobenius error <= 1e-9
  FP32  relative Frobenius error <= 1e-4
At the full adjoint workload size (8192 x 4096, k = 256, b = 64) the FP64 GPU
gradient is checked against central differences (h = 1e-6) of the FP64 GPU
forward map, and the FP32 gradient against the FP64 one.
"""
import numpy as np
import pytest
import torch

import inputs
from parity_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def _gpu_grad(rqb, A, G, k, b, dtype, seed=2):
    with rqb.Handle(dtype, max_rank=k, fixed_rank=True) as h:
        Ad = to_dev(A, dtype)
        Q, B, kk, rc = h.rqb_factor(Ad, 0.0, b, seed)
        assert rc == rqb.RQB_OK and kk == k
        dA = h.rqb_backward(to_dev(G, dtype))
        X = h.rqb_reconstruct(*A.shape)
        return to_np(dA), to_np(X)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-9), (torch.float32, 1e-4)])
@pytest.mark.parametrize("m,n,k,b", [(700, 500, 64, 16), (1037, 777, 96, 32), (512, 300, 40, 40)])
def test_backward_matches_oracle(orc, rqb_lib, dtype, tol, m, n, k, b):
    A, T, _ = inputs.config_adjoint_np(m=m, n=n, seed=m + n, rank=16, norm=10.0)
    prec = 64 if dtype == torch.float64 else 32
    if dtype == torch.float32:
        A = A.astype(np.float32).astype(np.float64)
    ro = orc.randqb_b(A, 0.0, b, seed=2, max_rank=k, fixed_rank=True, omega_prec=prec)
    Xo = ro.Q @ ro.B
    G = 2.0 * (Xo - T)
    if dtype == torch.float32:
        G = G.astype(np.float32).astype(np.float64)
    dA_o = orc.qqta_adjoint(A, ro.Q, ro.B, G, seed=2, omega_prec=prec)
    dA_g, X_g = _gpu_grad(rqb_lib, A, G, k, b, dtype)
    assert np.linalg.norm(X_g - Xo) <= (1e-11 if dtype == torch.float64 else 1e-5) * np.linalg.norm(A)
    assert np.linalg.norm(dA_g - dA_o) <= tol * np.linalg.norm(dA_o)


def test_autograd_function(orc, rqb_lib):
    m, n, k, b = 600, 400, 48, 16
    A, T, _ = inputs.config_adjoint_np(m=m, n=n, seed=5, rank=12, norm=10.0)
    At = to_dev(A, torch.float64).requires_grad_(True)
    Tt = to_dev(T, torch.float64)
    X = rqb_lib.qqta(At, k, b, seed=7)
    loss = ((X - Tt) ** 2).sum()
    loss.backward()
    ro = orc.randqb_b(A, 0.0, b, seed=7, max_rank=k, fixed_rank=True)
    G = 2.0 * (ro.Q @ ro.B - T)
    dA_o = orc.qqta_adjoint(A, ro.Q, ro.B, G, seed=7)
    assert abs(float(loss) - float(np.sum((ro.Q @ ro.B - T) ** 2))) <= 1e-10 * float(loss)
    assert np.linalg.norm(to_np(At.grad) - dA_o) <= 1e-9 * np.linalg.norm(dA_o)


def test_backward_full_size_central_differences(rqb_lib):
    """8192 x 4096, k = 256, b = 64: directional derivatives of L = ||Q Q^T A - T||^2."""
    m, n, k, b = 8192, 4096, 256, 64
    A, T, _ = inputs.config_adjoint_np(m=m, n=n, seed=5, rank=64, norm=10.0)
    Ad = to_dev(A, torch.float64)
    Td = to_dev(T, torch.float64)

    def loss(h, Adev):
        h.rqb_factor(Adev, 0.0, b, 3)
        X = h.rqb_reconstruct(m, n)
        return float(((X - Td) ** 2).sum()), X

    with rqb_lib.Handle(torch.float64, max_rank=k, fixed_rank=True) as h:
        L0, X0 = loss(h, Ad)
        G = rqb_lib.colmajor(2.0 * (X0 - Td))
        dA = h.rqb_backward(G).clone()
        gen = torch.Generator(device="cuda").manual_seed(11)
        hstep = 1e-6
        # FD noise is about u * L / h (~3e-3 here): use directions with a
        # component along the gradient so the derivative itself is large
        for _ in range(3):
            V = torch.randn(m, n, generator=gen, device="cuda", dtype=torch.float64)
            V = V / V.norm() + dA / dA.norm()
            V /= V.norm()
            Lp, _ = loss(h, rqb_lib.colmajor(Ad + hstep * V))
            Lm, _ = loss(h, rqb_lib.colmajor(Ad - hstep * V))
            fd = (Lp - Lm) / (2 * hstep)
            an = float((dA * V).sum())
            assert abs(fd - an) <= 1e-5 * max(abs(an), 1.0), (fd, an)
    with rqb_lib.Handle(torch.float32, max_rank=k, fixed_rank=True) as h32:
        A32 = to_dev(A, torch.float32)
        h32.rqb_factor(A32, 0.0, b, 3)
        dA32 = h32.rqb_backward(G.float())
        assert float((dA32.double() - dA).norm() / dA.norm()) <= 1e-3
