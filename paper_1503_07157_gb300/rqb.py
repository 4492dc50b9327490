"""Python binding of librqb.so (include/rqb.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module converts torch
tensors to pointers/leading dimensions, calls the C ABI entry point of the
same name, and wraps returned device buffers as torch tensor views (through
__cuda_array_interface__, no copy).  There is no CPU fallback: when the
library is missing or cannot be loaded, every call raises.

Matrices are column-major: a torch tensor M of shape (rows, cols) is passed
with leading dimension M.stride(1) and must have M.stride(0) == 1 (use
`colmajor(t)` to get such a tensor).
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librqb.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "rqb.h")

RQB_OK = 0
RQB_ERR_INVALID = 1
RQB_ERR_NONFINITE = 2
RQB_ERR_BREAKDOWN = 3
RQB_ERR_OOM = 4
RQB_ERR_TIMEOUT = 5
RQB_ERR_CUDA = 6
RQB_NOT_CONVERGED = 7
RQB_ERR_UNSUPPORTED = 8
RQB_ERR_SCRATCH_LIMIT = 9

RQB_F64, RQB_F32, RQB_BF16 = 0, 1, 2
RQB_PREC_NATIVE, RQB_PREC_TF32X3, RQB_PREC_BF16 = 0, 1, 2
RQB_MAX_TRACKED_BLOCKS = 512
RQB_FLAG_PHASE_TIMING = 1
RQB_FLAG_SKIP_INNER_ORTH = 2
RQB_FLAG_OMEGA_SMEM = 4
RQB_NUM_PHASES = 8
PHASES = ("sketch", "orth", "project", "downdate", "control")


class RqbError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class rqb_config(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("prec", ctypes.c_int32), ("max_rank", ctypes.c_int64),
                ("fixed_rank", ctypes.c_int32), ("power", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class rqb_stats(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("blocks", ctypes.c_int64), ("status", ctypes.c_int32),
                ("direct_tests", ctypes.c_int32), ("normA2", ctypes.c_double), ("eps", ctypes.c_double),
                ("E", ctypes.c_double * RQB_MAX_TRACKED_BLOCKS), ("D", ctypes.c_double * RQB_MAX_TRACKED_BLOCKS),
                ("kernel_launches", ctypes.c_int32), ("svd_sweeps", ctypes.c_int32),
                ("phase_ms", ctypes.c_double * RQB_NUM_PHASES), ("phase_calls", ctypes.c_int32 * RQB_NUM_PHASES),
                ("gram_fallbacks", ctypes.c_int32), ("tile_width", ctypes.c_int32),
                ("near_identity", ctypes.c_int32), ("fused_gram", ctypes.c_int32),
                ("pass1_fp32", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_LIB = None


def lib() -> ctypes.CDLL:
    """Load librqb.so (built by paper_1503_07157_gb300.build); raise if absent."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1503_07157_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, u64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        PP, Pi64, Pd = ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
        sig = {
            "rqb_create": [P, P],
            "rqb_destroy": [P],
            "rqb_factor": [P, P, i64, i64, i64, dbl, i64, u64, PP, Pi64, PP, Pi64, Pi64],
            "rqb_factor_host": [P, P, i64, i64, i64, dbl, i64, u64, P, i64, P, i64, Pi64],
            "rqb_get_stats": [P, P],
            "rqb_omega": [P, i64, i64, i64, u64, P, i64],
            "rqb_sketch": [P, P, i64, i64, i64, i64, i64, u64, P, i64, Pd],
            "rqb_orth": [P, P, i64, i64, i64, P, i64, i64, P, i64],
            "rqb_project": [P, P, i64, i64, i64, P, i64, i64, P, i64, Pd],
            "rqb_downdate_sketch": [P, P, i64, P, i64, P, i64, i64, i64, i64, P, i64, i64, i64, u64, P, i64, Pd],
            "rqb_sketch_noalloc": [ctypes.c_int32, P, i64, i64, i64, i64, i64, u64, P, i64, Pd, P],
            "rqb_reconstruct": [P, P, i64],
            "rqb_factor_batched": [P, i64, P, P, P, P, P, i64, u64, P, P, P, P, P, P],
            "rqb_backward": [P, P, i64, P, i64],
            "rqb_svd": [P, i64, P, i64, Pd, P, i64],
            "rqb_wait_selftest": [P, Pd],
            "rqb_fp64_recip_selftest": [P, i64, P, P, P],
            "rqb_inject_alloc_failure": [i64],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = i32
        L.rqb_status_string.argtypes = [i32]
        L.rqb_status_string.restype = ctypes.c_char_p
        _LIB = L
    return _LIB


def status_string(status: int) -> str:
    return lib().rqb_status_string(int(status)).decode()


def declared_symbols(header: str = HEADER) -> list[str]:
    """Names of the functions declared in include/rqb.h."""
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(rqb_\w+)\s*\(", text, flags=re.M)))


def _check(rc: int, where: str, ok=(RQB_OK,)) -> int:
    if rc not in ok:
        raise RqbError(rc, where)
    return rc


def colmajor(t: torch.Tensor) -> torch.Tensor:
    """Same values, column-major storage (stride(0) == 1)."""
    if t.dim() != 2:
        raise ValueError("expected a matrix")
    if t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.t().contiguous().t()


def _ld(t: torch.Tensor) -> int:
    if t.stride(0) != 1:
        raise ValueError("matrix must be column-major (stride(0) == 1); use colmajor()")
    return max(int(t.stride(1)), int(t.shape[0]), 1)


def _need(t: torch.Tensor, dtype: torch.dtype, what: str) -> None:
    """The library reads t as `dtype`: refuse a tensor of another element type."""
    if t.dtype != dtype:
        raise TypeError(f"{what}: expected {dtype}, got {t.dtype}")


def _dtype_code(dtype: torch.dtype) -> int:
    return {torch.float64: RQB_F64, torch.float32: RQB_F32, torch.bfloat16: RQB_BF16}[dtype]


class _CudaView:
    def __init__(self, ptr, shape, strides, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "strides": tuple(strides), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def _view(ptr: int, rows: int, cols: int, ld: int, dtype: torch.dtype, device) -> torch.Tensor:
    if rows == 0 or cols == 0 or not ptr:
        return torch.empty((rows, cols), dtype=dtype, device=device)
    es = torch.empty((), dtype=dtype).element_size()
    ts = {torch.float64: "<f8", torch.float32: "<f4"}[dtype]
    return torch.as_tensor(_CudaView(ptr, (rows, cols), (es, es * ld), ts), device=device)


@dataclass
class Stats:
    k: int
    blocks: int
    status: int
    direct_tests: int
    normA2: float
    eps: float
    E: list
    D: list
    kernel_launches: int
    phase_ms: list
    phase_calls: list
    gram_fallbacks: int = 0
    tile_width: int = 0
    near_identity: int = 0
    fused_gram: int = 0
    pass1_fp32: int = 0


class Handle:
    """Owns an rqb_handle on the current CUDA device and stream."""

    def __init__(self, dtype: torch.dtype = torch.float32, prec: int = RQB_PREC_NATIVE, max_rank: int = 0,
                 fixed_rank: bool = False, power: int = 0, stream: torch.cuda.Stream | None = None,
                 flags: int = 0):
        self.dtype = dtype
        self.out_dtype = torch.float64 if dtype == torch.float64 else torch.float32
        self.device = torch.device("cuda", torch.cuda.current_device())
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        cfg = rqb_config(_dtype_code(dtype), prec, max_rank, int(fixed_rank), power,
                         ctypes.c_void_p(s.cuda_stream), flags, 0)
        h = ctypes.c_void_p()
        _check(lib().rqb_create(ctypes.byref(h), ctypes.byref(cfg)), "rqb_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rqb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- randQB_b ----------------------------------------------------------
    def rqb_factor(self, A: torch.Tensor, eps: float, b: int, seed: int = 0, check: bool = True):
        """Returns (Q view m x k, B view k x n, k, status); views are valid until the next call."""
        _need(A, self.dtype, "rqb_factor A")
        m, n = A.shape
        Qp, Bp = ctypes.c_void_p(), ctypes.c_void_p()
        ldq, ldb, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        rc = lib().rqb_factor(self._h, ctypes.c_void_p(A.data_ptr()), m, n, _ld(A), float(eps), b, seed,
                              ctypes.byref(Qp), ctypes.byref(ldq), ctypes.byref(Bp), ctypes.byref(ldb),
                              ctypes.byref(k))
        if check:
            _check(rc, "rqb_factor", ok=(RQB_OK, RQB_NOT_CONVERGED))
        kk = int(k.value)
        self._last_shape = (m, n)
        Q = _view(Qp.value or 0, m, kk, int(ldq.value), self.out_dtype, self.device)
        B = _view(Bp.value or 0, kk, n, int(ldb.value), self.out_dtype, self.device)
        return Q, B, kk, rc

    def rqb_factor_host(self, A_host: torch.Tensor, eps: float, b: int, seed: int, Q_host: torch.Tensor,
                        B_host: torch.Tensor):
        _need(A_host, self.dtype, "rqb_factor_host A")
        _need(Q_host, self.out_dtype, "rqb_factor_host Q")
        _need(B_host, self.out_dtype, "rqb_factor_host B")
        m, n = A_host.shape
        k = ctypes.c_int64()
        rc = lib().rqb_factor_host(self._h, ctypes.c_void_p(A_host.data_ptr()), m, n, _ld(A_host), float(eps), b,
                                   seed, ctypes.c_void_p(Q_host.data_ptr()), _ld(Q_host),
                                   ctypes.c_void_p(B_host.data_ptr()), _ld(B_host), ctypes.byref(k))
        _check(rc, "rqb_factor_host", ok=(RQB_OK, RQB_NOT_CONVERGED))
        self._last_shape = (m, n)
        return int(k.value), rc

    def rqb_reconstruct(self, m: int, n: int) -> torch.Tensor:
        X = colmajor(torch.empty(n, m, dtype=self.out_dtype, device=self.device).t())
        _check(lib().rqb_reconstruct(self._h, ctypes.c_void_p(X.data_ptr()), _ld(X)), "rqb_reconstruct")
        return X

    def rqb_backward(self, G: torch.Tensor) -> torch.Tensor:
        m, n = G.shape
        G = colmajor(G.to(self.out_dtype))
        dA = colmajor(torch.empty(n, m, dtype=self.out_dtype, device=self.device).t())
        _check(lib().rqb_backward(self._h, ctypes.c_void_p(G.data_ptr()), _ld(G), ctypes.c_void_p(dA.data_ptr()),
                                  _ld(dA)), "rqb_backward")
        return dA

    def rqb_svd(self, r: int):
        """Rank-r SVD of the last factorization: (U m x r, S numpy (r,), Vt r x n, Jacobi sweeps)."""
        st = rqb_stats()
        _check(lib().rqb_get_stats(self._h, ctypes.byref(st)), "rqb_get_stats")
        m, n = self._last_shape
        U = colmajor(torch.empty(r, m, dtype=self.out_dtype, device=self.device).t())
        Vt = colmajor(torch.empty(n, r, dtype=self.out_dtype, device=self.device).t())
        S = (ctypes.c_double * r)()
        _check(lib().rqb_svd(self._h, r, ctypes.c_void_p(U.data_ptr()), _ld(U),
                             ctypes.cast(S, ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(Vt.data_ptr()),
                             _ld(Vt)), "rqb_svd")
        lib().rqb_get_stats(self._h, ctypes.byref(st))
        import numpy as np
        return U, np.array(S[:], dtype=np.float64), Vt, int(st.svd_sweeps)

    def rqb_wait_selftest(self):
        """Run the bounded-wait self-test: returns (status, waited_ms)."""
        w = ctypes.c_double()
        rc = lib().rqb_wait_selftest(self._h, ctypes.byref(w))
        return rc, float(w.value)

    def rqb_factor_batched(self, As: list, eps: list, b: int, seed: int = 0):
        """As: column-major FP32 device matrices.  Returns [(Q view, B view, k, status)]."""
        cnt = len(As)
        Ap = (ctypes.c_void_p * cnt)(*[ctypes.c_void_p(a.data_ptr()) for a in As])
        mm = (ctypes.c_int64 * cnt)(*[a.shape[0] for a in As])
        nn = (ctypes.c_int64 * cnt)(*[a.shape[1] for a in As])
        ld = (ctypes.c_int64 * cnt)(*[_ld(a) for a in As])
        ee = (ctypes.c_double * cnt)(*[float(e) for e in eps])
        Qp, Bp = (ctypes.c_void_p * cnt)(), (ctypes.c_void_p * cnt)()
        lq, lb, kk = (ctypes.c_int64 * cnt)(), (ctypes.c_int64 * cnt)(), (ctypes.c_int64 * cnt)()
        st = (ctypes.c_int * cnt)()
        _check(lib().rqb_factor_batched(self._h, cnt, Ap, mm, nn, ld, ee, b, seed, Qp, lq, Bp, lb, kk, st),
               "rqb_factor_batched")
        out = []
        for t in range(cnt):
            k = int(kk[t])
            out.append((_view(Qp[t] or 0, mm[t], k, int(lq[t]), torch.float32, self.device),
                        _view(Bp[t] or 0, k, nn[t], int(lb[t]), torch.float32, self.device), k, int(st[t])))
        return out

    def rqb_get_stats(self) -> Stats:
        st = rqb_stats()
        _check(lib().rqb_get_stats(self._h, ctypes.byref(st)), "rqb_get_stats")
        nb = min(int(st.blocks), RQB_MAX_TRACKED_BLOCKS)
        return Stats(int(st.k), int(st.blocks), int(st.status), int(st.direct_tests), float(st.normA2),
                     float(st.eps), list(st.E[:nb]), list(st.D[:nb]), int(st.kernel_launches),
                     list(st.phase_ms), list(st.phase_calls), int(st.gram_fallbacks), int(st.tile_width),
                     int(st.near_identity), int(st.fused_gram),
                     int(st.pass1_fp32))

    # -- steps ---------------------------------------------------------------
    def rqb_omega(self, n: int, col0: int, ncols: int, seed: int) -> torch.Tensor:
        out = colmajor(torch.empty(ncols, n, dtype=self.out_dtype, device=self.device).t())
        _check(lib().rqb_omega(self._h, n, col0, ncols, seed, ctypes.c_void_p(out.data_ptr()), _ld(out)),
               "rqb_omega")
        return out

    def rqb_sketch(self, A: torch.Tensor, col0: int, ncols: int, seed: int):
        _need(A, self.dtype, "rqb_sketch A")
        m, n = A.shape
        Y = colmajor(torch.empty(ncols, m, dtype=self.out_dtype, device=self.device).t())
        nrm = ctypes.c_double()
        _check(lib().rqb_sketch(self._h, ctypes.c_void_p(A.data_ptr()), m, n, _ld(A), col0, ncols, seed,
                                ctypes.c_void_p(Y.data_ptr()), _ld(Y), ctypes.byref(nrm)), "rqb_sketch")
        return Y, float(nrm.value)

    def rqb_orth(self, Y: torch.Tensor, Qbar: torch.Tensor | None):
        _need(Y, self.out_dtype, "rqb_orth Y")
        if Qbar is not None:
            _need(Qbar, self.out_dtype, "rqb_orth Qbar")
        m, p = Y.shape
        Qi = colmajor(torch.empty(p, m, dtype=self.out_dtype, device=self.device).t())
        if Qbar is None or Qbar.shape[1] == 0:
            qp, kprev, ldqb = ctypes.c_void_p(0), 0, m
        else:
            qp, kprev, ldqb = ctypes.c_void_p(Qbar.data_ptr()), Qbar.shape[1], _ld(Qbar)
        rc = lib().rqb_orth(self._h, ctypes.c_void_p(Y.data_ptr()), m, p, _ld(Y), qp, kprev, ldqb,
                            ctypes.c_void_p(Qi.data_ptr()), _ld(Qi))
        _check(rc, "rqb_orth")
        return Qi

    def rqb_project(self, Qi: torch.Tensor, A: torch.Tensor):
        _need(Qi, self.out_dtype, "rqb_project Qi")
        _need(A, self.dtype, "rqb_project A")
        m, p = Qi.shape
        n = A.shape[1]
        Bi = colmajor(torch.empty(n, p, dtype=self.out_dtype, device=self.device).t())
        nrm = ctypes.c_double()
        _check(lib().rqb_project(self._h, ctypes.c_void_p(Qi.data_ptr()), m, p, _ld(Qi),
                                 ctypes.c_void_p(A.data_ptr()), n, _ld(A), ctypes.c_void_p(Bi.data_ptr()), _ld(Bi),
                                 ctypes.byref(nrm)), "rqb_project")
        return Bi, float(nrm.value)

    def rqb_downdate_sketch(self, A: torch.Tensor, Qi: torch.Tensor, Bi: torch.Tensor, W: torch.Tensor, col0: int,
                            ncols: int, seed: int):
        _need(A, self.dtype, "rqb_downdate_sketch A")
        _need(W, self.dtype, "rqb_downdate_sketch W")
        _need(Qi, self.out_dtype, "rqb_downdate_sketch Qi")
        _need(Bi, self.out_dtype, "rqb_downdate_sketch Bi")
        m, n = A.shape
        p = Qi.shape[1]
        Y = colmajor(torch.empty(ncols, m, dtype=self.out_dtype, device=self.device).t())
        nrm = ctypes.c_double()
        _check(lib().rqb_downdate_sketch(self._h, ctypes.c_void_p(A.data_ptr()), _ld(A),
                                         ctypes.c_void_p(Qi.data_ptr()), _ld(Qi), ctypes.c_void_p(Bi.data_ptr()),
                                         _ld(Bi), m, n, p, ctypes.c_void_p(W.data_ptr()), _ld(W), col0, ncols, seed,
                                         ctypes.c_void_p(Y.data_ptr()), _ld(Y), ctypes.byref(nrm)),
               "rqb_downdate_sketch")
        return Y, float(nrm.value)


def rqb_sketch_noalloc(A: torch.Tensor, col0: int, ncols: int, seed: int, Y: torch.Tensor,
                       stream: torch.cuda.Stream | None = None, want_norm: bool = True):
    """Y (caller-allocated, m x ncols, column-major) = A Omega(:, col0:col0+ncols)
    without any device allocation inside the library; returns (status, ||A||_F^2 or None)."""
    m, n = A.shape
    s = stream if stream is not None else torch.cuda.current_stream()
    nrm = ctypes.c_double()
    rc = lib().rqb_sketch_noalloc(_dtype_code(A.dtype), ctypes.c_void_p(A.data_ptr()), m, n, _ld(A), col0, ncols,
                                  seed, ctypes.c_void_p(Y.data_ptr()), _ld(Y),
                                  ctypes.byref(nrm) if want_norm else None, ctypes.c_void_p(s.cuda_stream))
    return rc, (float(nrm.value) if want_norm else None)


def rqb_fp64_recip_selftest(x: torch.Tensor):
    """(1/x, 1/sqrt(x)) of a CUDA FP64 vector through the library's Newton
    reciprocal and reciprocal square root (the Cholesky pivots' helpers)."""
    x = x.contiguous()
    rcp, rsq = torch.empty_like(x), torch.empty_like(x)
    _check(lib().rqb_fp64_recip_selftest(ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(rcp.data_ptr()),
                                         ctypes.c_void_p(rsq.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
           "rqb_fp64_recip_selftest")
    return rcp, rsq


class QQtA(torch.autograd.Function):
    """X = Q Q^T A with Q from fixed-rank randQB_b (k = max_rank, Omega from
    `seed`); backward through rqb_backward.  Each call owns a handle, so
    several nodes of one graph do not share factorization state."""

    @staticmethod
    def forward(ctx, A: torch.Tensor, k: int, b: int, seed: int):
        A = colmajor(A.detach())
        h = Handle(A.dtype, max_rank=k, fixed_rank=True)
        h.rqb_factor(A, 0.0, b, seed)
        X = h.rqb_reconstruct(*A.shape)
        ctx.save_for_backward(A)
        ctx.h = h
        return X

    @staticmethod
    def backward(ctx, G: torch.Tensor):
        dA = ctx.h.rqb_backward(G)
        return dA, None, None, None


def qqta(A: torch.Tensor, k: int, b: int, seed: int = 0) -> torch.Tensor:
    """Differentiable fixed-rank approximation Q Q^T A (Omega held fixed)."""
    return QQtA.apply(A, k, b, seed)
