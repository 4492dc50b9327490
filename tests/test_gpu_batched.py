"""rqb_factor_batched: many FP32 matrices of uneven sizes in one graph launch
(a device-side block loop; tile width picked by the autotuner).

Each matrix is compared with the oracle (randQB_b, same seed, binary32 Omega):
rank exact (or one block away inside the decision band), |r_gpu - r_orc| <=
1e-5 ||A_t||_F, ||Q^T Q - I||_max <= 1e-5; a matrix with a NaN reports
RQB_ERR_NONFINITE without affecting the others; results equal those of the
single-matrix entry point on the same inputs (same rank, residuals within 1e-5).
"""
import numpy as np
import pytest
import torch

import inputs
from parity_util import assert_residual_parity, check_rank, oracle_at_rank, orth_err, resid, to_dev, to_np

pytestmark = pytest.mark.gpu


def _batch(seed=0):
    rng = np.random.default_rng(seed)
    mats = []
    shapes = [(900, 600, 40), (257, 129, 10), (513, 513, 25), (64, 300, 8), (5, 3, 2), (1000, 33, 30),
              (777, 400, 60), (300, 299, 5), (128, 128, 12), (640, 480, 20), (33, 31, 15), (1500, 700, 50)]
    for i, (m, n, r) in enumerate(shapes):
        s = inputs.spectrum_exp(min(m, n), r)
        A = inputs.usv(m, n, s, seed=100 + i).astype(np.float32).astype(np.float64)
        eps = (1e-3 if i % 2 == 0 else 1e-2) * np.linalg.norm(A)
        mats.append((A, eps))
    return mats


@pytest.mark.parametrize("b", [32, 20])
def test_batched_matches_oracle(orc, rqb_lib, b):
    mats = _batch()
    devs = [to_dev(A, torch.float32) for A, _ in mats]
    with rqb_lib.Handle(torch.float32) as h:
        out = h.rqb_factor_batched(devs, [e for _, e in mats], b, seed=9)
        res = [(to_np(Q), to_np(B), k, st) for Q, B, k, st in out]
    for (A, eps), (Q, B, k, st) in zip(mats, res):
        ro = orc.randqb_b(A, eps, b, seed=9, omega_prec=32)
        nA = np.linalg.norm(A)
        assert st in (rqb_lib.RQB_OK, rqb_lib.RQB_NOT_CONVERGED), st
        check_rank(k, ro, eps, b, rel_band=1e-3)
        rk = oracle_at_rank(orc, A, ro, k, b, 9, omega_prec=32)
        assert_residual_parity(A, Q, B, rk, 1e-5, b=b, eps=eps if st == rqb_lib.RQB_OK else None)
        if st == rqb_lib.RQB_OK:
            assert resid(A, Q, B) <= eps * (1 + 1e-4)
        assert orth_err(Q) <= 1e-5


def test_batched_equals_single(rqb_lib):
    mats = _batch(seed=1)[:6]
    devs = [to_dev(A, torch.float32) for A, _ in mats]
    with rqb_lib.Handle(torch.float32) as h:
        out = h.rqb_factor_batched(devs, [e for _, e in mats], 32, seed=4)
        res = [(to_np(Q), to_np(B), k, st) for Q, B, k, st in out]
    with rqb_lib.Handle(torch.float32) as h1:
        for (A, eps), d, (Q, B, k, st) in zip(mats, devs, res):
            Q1, B1, k1, rc1 = h1.rqb_factor(d, eps, 32, 4, check=False)
            assert k1 == k and rc1 == st
            assert abs(resid(A, Q, B) - resid(A, to_np(Q1), to_np(B1))) <= 1e-5 * np.linalg.norm(A)


def test_batched_nonfinite_isolated(rqb_lib):
    mats = _batch(seed=2)[:4]
    A_bad = mats[1][0].copy()
    A_bad[3, 2] = np.nan
    mats[1] = (A_bad, mats[1][1])
    devs = [to_dev(A, torch.float32) for A, _ in mats]
    with rqb_lib.Handle(torch.float32) as h:
        out = h.rqb_factor_batched(devs, [e for _, e in mats], 32, seed=4)
    sts = [st for _, _, _, st in out]
    assert sts[1] == rqb_lib.RQB_ERR_NONFINITE
    assert all(s == rqb_lib.RQB_OK for i, s in enumerate(sts) if i != 1)


def test_batched_rejects_bad_arguments(rqb_lib):
    with rqb_lib.Handle(torch.float64) as h:
        A = to_dev(np.ones((8, 4)), torch.float64)
        with pytest.raises(rqb_lib.RqbError) as e:
            h.rqb_factor_batched([A], [1.0], 4)
        assert e.value.status == rqb_lib.RQB_ERR_UNSUPPORTED
    with rqb_lib.Handle(torch.float32) as h:
        A = to_dev(np.ones((8, 4)), torch.float32)
        with pytest.raises(rqb_lib.RqbError):
            h.rqb_factor_batched([A], [1.0], 33)


def test_batched_zero_matrix_empty_factorization(rqb_lib):
    """A zero matrix (||A|| = 0 <= eps) in the batch gets k = 0 and RQB_OK; the
    others are unaffected."""
    mats = _batch(seed=3)[:3]
    m0, n0 = mats[1][0].shape
    mats[1] = (np.zeros((m0, n0)), 0.0)
    devs = [to_dev(A, torch.float32) for A, _ in mats]
    with rqb_lib.Handle(torch.float32) as h:
        out = h.rqb_factor_batched(devs, [e for _, e in mats], 32, seed=4)
        # the factors live in the handle's buffers: read them before it closes
        fac = [(to_np(Q), to_np(B), k, st) for Q, B, k, st in out]
    assert fac[1][2] == 0 and fac[1][3] == rqb_lib.RQB_OK
    for i in (0, 2):
        Q, B, k, st = fac[i]
        assert st == rqb_lib.RQB_OK and k > 0
        assert resid(mats[i][0], Q, B) <= mats[i][1] * (1 + 1e-4)


def _run(rqb_lib, mats, eps, b=32, seed=4):
    devs = [to_dev(A, torch.float32) for A, _ in mats] if not torch.is_tensor(mats[0]) else mats
    with rqb_lib.Handle(torch.float32) as h:
        out = h.rqb_factor_batched(devs, eps, b, seed=seed)
        res = [(to_np(Q), to_np(B), k, st) for Q, B, k, st in out]
        out2 = h.rqb_factor_batched(devs, eps, b, seed=seed)      # the cached graph
        res2 = [(to_np(Q), to_np(B), k, st) for Q, B, k, st in out2]
        stats = h.rqb_get_stats()
    return res, res2, stats


def test_batched_one_graph_reused_and_autotuned(rqb_lib, tmp_path, monkeypatch):
    """The whole batch runs as one graph launch whose block loop is a WHILE
    node: the launch count is the prologue plus 14 kernels per block, a
    second call reuses the graph with bit-identical results, and the
    autotuner writes its choice for the batch class to RQB_AUTOTUNE_CACHE."""
    mats = _batch(seed=5)
    eps = [e for _, e in mats]
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("RQB_AUTOTUNE_CACHE", str(cache))
    res, res2, st = _run(rqb_lib, mats, eps)
    for (Q, B, k, s), (Q2, B2, k2, s2) in zip(res, res2):
        assert k == k2 and s == s2
        assert np.array_equal(Q, Q2) and np.array_equal(B, B2)
    lines = cache.read_text().split("\n")
    lines = [l for l in lines if l]
    assert len(lines) == 1 and lines[0].startswith("batched_projection_width ")
    width = int(lines[0].split()[-1])
    assert width in (128, 256) and st.tile_width == width
    max_k = max(k for _, _, k, _ in res)
    blocks = -(-max_k // 32)
    assert (st.kernel_launches - 3) % 14 == 0 and (st.kernel_launches - 3) // 14 >= blocks
    # a new handle (a new process alike) reads the choice instead of tuning again
    res3, _, st3 = _run(rqb_lib, mats, eps)
    assert len([l for l in cache.read_text().split("\n") if l]) == 1 and st3.tile_width == width
    for (Q, B, k, s), (Q3, B3, k3, s3) in zip(res, res3):
        assert k == k3 and np.array_equal(Q, Q3) and np.array_equal(B, B3)


def test_batched_projection_widths_bitwise_equal(rqb_lib, tmp_path, monkeypatch):
    """Each B_i entry is one thread's sum over the rows in the same order
    whatever the projection's tile width, so both widths the autotuner picks
    from give the same factors bit for bit."""
    mats = _batch(seed=6)[:8]
    eps = [e for _, e in mats]
    tune = tmp_path / "tune.txt"
    monkeypatch.setenv("RQB_AUTOTUNE_CACHE", str(tune))
    _run(rqb_lib, mats, eps)
    key = tune.read_text().split()[1]
    out = {}
    for w in (128, 256):
        f = tmp_path / f"w{w}.txt"
        f.write_text(f"batched_projection_width {key} {w}\n")
        monkeypatch.setenv("RQB_AUTOTUNE_CACHE", str(f))
        res, _, st = _run(rqb_lib, mats, eps)
        assert st.tile_width == w
        out[w] = res
    for (Q1, B1, k1, s1), (Q2, B2, k2, s2) in zip(out[128], out[256]):
        assert k1 == k2 and s1 == s2
        assert np.array_equal(Q1, Q2) and np.array_equal(B1, B2)
