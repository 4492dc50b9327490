"""CPU FP64 oracle for blocked randomized QB (Martinsson & Voronin, arXiv:1503.07157).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg import this package.  The product library never does.

Thin ctypes wrapper over oracle/librqb_oracle.so (built from rqb_oracle.c);
arrays are numpy float64, column-major (Fortran order).

Functions and the passages they follow:
  philox4x32_10  -- the counter-based generator of Salmon et al. (SC'11)
  omega          -- Fig. randQB_b line (2), Omega_i = randn(n, b), indexed by
                    global column so that blocks slice one Omega (eq. OmegaBlock);
                    prec 64, 32, 19 (binary32 draw rounded to TF32) or 8
                    (rounded to BF16)
  round_tf32     -- rounding to 11 significant bits, ties away from zero
  round_bf16     -- rounding to 8 significant bits, ties to even
  orth           -- Sec. 2.4, unpivoted Householder QR with diag(R) >= 0
  sketch         -- Fig. randQB_b line (3), A Omega_i
  orth_reproject -- Fig. randQB_b lines (3) and (3')
  randqb_b       -- Fig. randQB_b (power > 0: Fig. randQB_pb; skip_inner_orth:
                    the Sec. 5.4 variant; storage_prec 16: the residual kept
                    in BF16, stopping on its direct norm)
  randqb         -- Fig. randQB (unblocked)
  svd_values     -- singular values by one-sided Jacobi (for the Eckart-Young
                    bound of eq. minerrors on small inputs)
  qqta_adjoint   -- gradient through the fixed-rank map A -> Q Q^T A with Omega
                    held fixed (derived from the projector onto R(A Omega),
                    Sec. 4.1 / Prop. 4.1(c)); the paper itself has no derivatives
"""
import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64, u64, dbl, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        P = ctypes.c_void_p
        lib.orc_philox4x32_10.argtypes = [P, P, P]
        lib.orc_omega.argtypes = [u64, ctypes.c_uint32, i64, i64, i64, i32, P, i64]
        lib.orc_orth.argtypes = [P, i64, i64, i64, P, i64, P, i64]
        lib.orc_randqb_b.argtypes = [P, i64, i64, i64, dbl, i64, u64, i64, i32, i32, i32, i32,
                                     P, i64, P, i64, P]
        lib.orc_randqb_b.restype = i32
        lib.orc_randqb.argtypes = [P, i64, i64, i64, i64, u64, i32, P, i64, P, i64]
        lib.orc_randqb.restype = i32
        lib.orc_svd_values.argtypes = [P, i64, i64, i64, P]
        lib.orc_sketch.argtypes = [P, i64, i64, i64, u64, i64, i64, i32, P, i64]
        lib.orc_orth_reproject.argtypes = [P, i64, i64, i64, P, i64, i64, P, i64]
        lib.orc_num_threads.restype = i32
        lib.orc_qqta_adjoint.argtypes = [P, i64, i64, i64, P, i64, P, i64, i64, u64, i32, P, i64, P, i64]
        lib.orc_qqta_adjoint.restype = i32
        lib.orc_round_tf32.argtypes = [dbl]
        lib.orc_round_tf32.restype = dbl
        lib.orc_round_bf16.argtypes = [dbl]
        lib.orc_round_bf16.restype = dbl
        lib.orc_round_bf16_n.argtypes = [P, P, i64]
        lib.orc_rsvd.argtypes = [P, i64, i64, i64, P, i64, i64, i64, P, i64, P, P, i64]
        lib.orc_rsvd.restype = i32
        lib.orc_randqb_b_store.argtypes = [P, i64, i64, i64, dbl, i64, u64, i64, i32, i32, i32, i32, i32,
                                           P, i64, P, i64, P]
        lib.orc_randqb_b_store.restype = i32
        _LIB = lib
    return _LIB


class _Res(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("blocks", ctypes.c_int64), ("status", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("normA2", ctypes.c_double),
                ("E", ctypes.c_void_p), ("D", ctypes.c_void_p), ("max_blocks", ctypes.c_int64)]


def _f64(a):
    return np.asfortranarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_lib().orc_num_threads())


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def round_tf32(x: float) -> float:
    return float(_lib().orc_round_tf32(float(x)))


def round_bf16(x: float) -> float:
    return float(_lib().orc_round_bf16(float(x)))


def round_bf16_array(x) -> np.ndarray:
    """Elementwise round_bf16 of an array (same shape, float64)."""
    a = np.array(x, dtype=np.float64, order="F", copy=True)
    _lib().orc_round_bf16_n(_ptr(a), _ptr(a), a.size)
    return a


def omega(seed: int, n: int, col0: int, ncols: int, prec: int = 64, stream: int = 0):
    out = np.zeros((n, ncols), dtype=np.float64, order="F")
    _lib().orc_omega(seed, stream, n, col0, ncols, prec, _ptr(out), n)
    return out


def orth(Y, return_r: bool = False):
    Y = _f64(Y)
    m, p = Y.shape
    Q = np.zeros((m, p), order="F")
    R = np.zeros((p, p), order="F")
    _lib().orc_orth(_ptr(Y), m, p, m, _ptr(Q), m, _ptr(R), p)
    return (Q, R) if return_r else Q


def sketch(A, seed: int, col0: int, p: int, omega_prec: int = 64, lda_pad: int = 0, ldy_pad: int = 0):
    """A Omega(:, col0 : col0 + p).  lda_pad / ldy_pad > 0 place A and Y in
    taller buffers (leading dims m + pad) to exercise the strided forms."""
    A = _f64(A)
    m, n = A.shape
    lda, ldy = m + lda_pad, m + ldy_pad
    if lda_pad:
        Abuf = np.zeros((lda, n), order="F")
        Abuf[:m, :] = A
    else:
        Abuf = A
    Ybuf = np.full((ldy, p), np.nan, order="F")
    _lib().orc_sketch(_ptr(Abuf), m, n, lda, seed, col0, p, omega_prec, _ptr(Ybuf), ldy)
    if ldy_pad and not np.all(np.isnan(Ybuf[m:, :])):
        raise AssertionError("orc_sketch wrote past row m of a strided Y")
    return Ybuf[:m, :].copy(order="F")


def orth_reproject(Y, Qbar, ld_pad: int = 0):
    """Lines (3), (3').  ld_pad > 0 places Y, Qbar and Q_i in taller buffers
    (leading dims m + pad) to exercise the strided forms."""
    Y = _f64(Y)
    m, p = Y.shape
    Qbar = _f64(Qbar) if Qbar is not None and Qbar.shape[1] > 0 else np.zeros((m, 0), order="F")
    kprev = Qbar.shape[1]
    ld = m + ld_pad
    Ybuf = np.zeros((ld, p), order="F")
    Ybuf[:m, :] = Y
    qb = np.zeros((ld, max(kprev, 1)), order="F")
    qb[:m, :kprev] = Qbar
    Qi = np.full((ld, p), np.nan, order="F")
    _lib().orc_orth_reproject(_ptr(Ybuf), m, p, ld, _ptr(qb), kprev, ld, _ptr(Qi), ld)
    if ld_pad and not np.all(np.isnan(Qi[m:, :])):
        raise AssertionError("orc_orth_reproject wrote past row m of a strided Q_i")
    return Qi[:m, :].copy(order="F")


@dataclass
class QBResult:
    Q: np.ndarray
    B: np.ndarray
    k: int
    blocks: int
    status: int
    normA2: float
    E: np.ndarray = field(repr=False)   # running downdate after each block
    D: np.ndarray = field(repr=False)   # direct ||A^(i)||_F^2 after each block

    def residual_downdate(self) -> float:
        return float(np.sqrt(max(self.E[-1], 0.0)))

    def residual_direct(self) -> float:
        return float(np.sqrt(self.D[-1]))


def randqb_b(A, eps: float, b: int, seed: int = 0, max_rank: int = 0, fixed_rank: bool = False,
             power: int = 0, skip_inner_orth: bool = False, omega_prec: int = 64, storage_prec: int = 64) -> QBResult:
    A = _f64(A)
    m, n = A.shape
    rmax = min(m, n)
    kcap = rmax if (max_rank <= 0 or max_rank > rmax) else max_rank
    Q = np.zeros((m, kcap), order="F")
    B = np.zeros((kcap, n), order="F")
    nbmax = (kcap + b - 1) // b + 1
    E = np.zeros(nbmax)
    D = np.zeros(nbmax)
    res = _Res(0, 0, 0, 0, 0.0, E.ctypes.data, D.ctypes.data, nbmax)
    rc = _lib().orc_randqb_b_store(_ptr(A), m, n, m, float(eps), b, seed, kcap, int(fixed_rank),
                                   int(power), int(skip_inner_orth), int(omega_prec), int(storage_prec),
                                   _ptr(Q), m, _ptr(B), kcap, ctypes.byref(res))
    if rc != 0:
        raise ValueError("orc_randqb_b: invalid arguments")
    k, s = int(res.k), int(res.blocks)
    return QBResult(Q=Q[:, :k].copy(order="F"), B=B[:k, :].copy(order="F"), k=k, blocks=s,
                    status=int(res.status), normA2=float(res.normA2), E=E[:s].copy(), D=D[:s].copy())


def randqb(A, l: int, seed: int = 0, omega_prec: int = 64):
    A = _f64(A)
    m, n = A.shape
    Q = np.zeros((m, l), order="F")
    B = np.zeros((l, n), order="F")
    rc = _lib().orc_randqb(_ptr(A), m, n, m, l, seed, omega_prec, _ptr(Q), m, _ptr(B), l)
    if rc != 0:
        raise ValueError("orc_randqb: invalid arguments")
    return Q, B


def svd_values(A):
    A = _f64(A)
    m, n = A.shape
    s = np.zeros(min(m, n))
    _lib().orc_svd_values(_ptr(A), m, n, m, _ptr(s))
    return s


def rsvd(Q, B, r: int):
    """Rank-r SVD of Q B (Sec. 2): returns U (m x r), S (r,), Vt (r x n)."""
    Q, B = _f64(Q), _f64(B)
    m, k = Q.shape
    n = B.shape[1]
    U = np.zeros((m, r), order="F")
    S = np.zeros(r)
    Vt = np.zeros((r, n), order="F")
    rc = _lib().orc_rsvd(_ptr(Q), m, k, m, _ptr(B), n, k, r, _ptr(U), m, _ptr(S), _ptr(Vt), r)
    if rc != 0:
        raise ValueError("orc_rsvd: invalid arguments")
    return U, S, Vt


def qqta_adjoint(A, Q, B, G, seed: int = 0, omega_prec: int = 64):
    """dL/dA for X = Q Q^T A (fixed Omega) given G = dL/dX and the forward's Q, B."""
    A, Q, B, G = _f64(A), _f64(Q), _f64(B), _f64(G)
    m, n = A.shape
    k = Q.shape[1]
    dA = np.zeros((m, n), order="F")
    rc = _lib().orc_qqta_adjoint(_ptr(A), m, n, m, _ptr(Q), m, _ptr(B), k, k, seed, omega_prec,
                                 _ptr(G), m, _ptr(dA), m)
    if rc != 0:
        raise ValueError("orc_qqta_adjoint: singular B Omega or bad rank")
    return dA
