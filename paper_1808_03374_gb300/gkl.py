"""Thin Python binding of the C ABI in include/gkl.h (ctypes).

Argument marshalling only: every step of the computation runs in libgkl's CUDA
kernels.  PyTorch supplies device memory and the current stream.  If the
library is missing the import of this module fails loudly; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from .build import LIB as _LIB_PATH

FP64, FP32, BLOCK, BLOCK16 = 0, 1, 2, 3
REORTH_FULL, REORTH_PARTIAL, REORTH_DGKS, REORTH_ONESIDED = 0, 1, 2, 3
OK, ERR_ARG, ERR_CUDA, ERR_NONFINITE, NOT_CONVERGED, ERR_GAP, ERR_STATE, RANK_DEFICIENT = range(8)

_PREC = {"fp64": FP64, "fp32": FP32, "block": BLOCK, "block16": BLOCK16}
_REORTH = {"full": REORTH_FULL, "partial": REORTH_PARTIAL, "dgks": REORTH_DGKS, "onesided": REORTH_ONESIDED}
_DTYPE = {FP64: torch.float64, FP32: torch.float32, BLOCK: torch.float32, BLOCK16: torch.float32}

EXPORTS = ["gkl_version", "gkl_last_error", "gkl_opts_default", "gkl_colstats", "gkl_init", "gkl_set_stream",
           "gkl_set_weights", "gkl_matvec", "gkl_rmatvec", "gkl_svd", "gkl_destroy", "gkl_matvec_noalloc",
           "gkl_grad", "gkl_matmat", "gkl_scores", "gkl_sync"]


class GKLError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gkl error {code}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("ell", ctypes.c_int32), ("k_keep", ctypes.c_int32),
                ("reorth", ctypes.c_int32), ("precision", ctypes.c_int32), ("maxit", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("block", ctypes.c_int32), ("out_host", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("tol", ctypes.c_double), ("omega", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("v0", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("matvec_pairs", ctypes.c_int64), ("restarts", ctypes.c_int32), ("cycles", ctypes.c_int32),
                ("reorth_u", ctypes.c_int32), ("reorth_v", ctypes.c_int32), ("breakdowns", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("max_rel_resid", ctypes.c_double), ("dtheta1", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("launches", ctypes.c_int64), ("n_mv", ctypes.c_int64),
                ("n_rmv", ctypes.c_int64), ("ms_mv", ctypes.c_double), ("ms_rmv", ctypes.c_double),
                ("jacobi_sweeps", ctypes.c_int32), ("svd_fallbacks", ctypes.c_int32),
                ("svd_clusters", ctypes.c_int32), ("rank", ctypes.c_int32), ("ms_svd", ctypes.c_double),
                ("ms_cgs", ctypes.c_double), ("second_u", ctypes.c_int32), ("second_v", ctypes.c_int32),
                ("refine_cycles", ctypes.c_int32), ("reserved1", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def library_path() -> str:
    return _LIB_PATH


def load(path: str | None = None) -> ctypes.CDLL:
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libgkl.so is not built ({path}); run paper_1808_03374_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.gkl_version.restype = ctypes.c_char_p
    lib.gkl_last_error.restype = ctypes.c_char_p
    lib.gkl_last_error.argtypes = [vp]
    lib.gkl_opts_default.argtypes = [ctypes.POINTER(Opts)]
    lib.gkl_opts_default.restype = None
    lib.gkl_colstats.argtypes = [vp, i64, i64, i64, vp, vp, vp, vp]
    lib.gkl_init.argtypes = [ctypes.POINTER(vp), vp, i64, i64, i64, vp, vp, vp]
    lib.gkl_set_stream.argtypes = [vp, vp]
    lib.gkl_set_weights.argtypes = [vp, vp, vp]
    lib.gkl_matvec.argtypes = [vp, i32, vp, vp]
    lib.gkl_rmatvec.argtypes = [vp, i32, vp, vp]
    lib.gkl_svd.argtypes = [vp, ctypes.POINTER(Opts), vp, vp, vp, vp, ctypes.POINTER(Info)]
    lib.gkl_destroy.argtypes = [vp]
    lib.gkl_matvec_noalloc.argtypes = [vp, i64, i64, i64, vp, vp, i32, vp, vp, vp]
    lib.gkl_grad.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double]
    lib.gkl_grad.restype = ctypes.c_int
    lib.gkl_matmat.argtypes = [vp, i32, i32, i32, vp, i64, vp, i64]
    lib.gkl_matmat.restype = ctypes.c_int
    lib.gkl_scores.argtypes = [vp, vp, i32]
    lib.gkl_sync.argtypes = [vp]
    for f in ("gkl_colstats", "gkl_init", "gkl_set_stream", "gkl_set_weights", "gkl_matvec", "gkl_rmatvec",
              "gkl_svd", "gkl_destroy", "gkl_matvec_noalloc", "gkl_scores", "gkl_sync"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


_LIB = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(code: int, h=None):
    if code != OK:
        raise GKLError(code, lib().gkl_last_error(h).decode())


def _need_buffer(t, shape, dtype=None, cuda=None, what="buffer"):
    """Raise ValueError unless tensor t has exactly this shape (and dtype,
    device kind), contiguous: the library takes its sizes from the handle, so a
    smaller buffer would be read or written past its end."""
    if tuple(t.shape) != tuple(shape) and not (len(shape) == 1 and t.numel() == shape[0] and t.dim() <= 1):
        raise ValueError(f"{what}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{what}: expected dtype {dtype}, got {t.dtype}")
    if cuda is not None and t.is_cuda != cuda:
        raise ValueError(f"{what}: expected {'device' if cuda else 'host'} memory")
    if not t.is_contiguous():
        raise ValueError(f"{what}: must be contiguous")


def colstats(packed: torch.Tensor, n: int):
    """Per-SNP mean, 1/SD and observed count of a packed matrix (device tensors)."""
    assert packed.is_cuda and packed.dtype == torch.uint8 and packed.dim() == 2 and packed.is_contiguous()
    m, stride = packed.shape
    mu = torch.empty(m, dtype=torch.float64, device=packed.device)
    sc = torch.empty(m, dtype=torch.float64, device=packed.device)
    nobs = torch.empty(m, dtype=torch.int64, device=packed.device)
    _check(lib().gkl_colstats(_ptr(packed), n, m, stride, _ptr(mu), _ptr(sc), _ptr(nobs), _stream()))
    return mu, sc, nobs


@dataclass
class SVDResult:
    sigma: np.ndarray
    U: torch.Tensor | None
    V: torch.Tensor | None
    resid: np.ndarray
    info: dict
    status: int

    @property
    def converged(self) -> bool:
        return self.status in (OK, RANK_DEFICIENT)


class GKL:
    """Handle over a packed genotype matrix resident on the GPU (borrowed)."""

    def __init__(self, packed: torch.Tensor, n: int, mu: torch.Tensor | None = None,
                 scale: torch.Tensor | None = None):
        assert packed.is_cuda and packed.dtype == torch.uint8 and packed.dim() == 2 and packed.is_contiguous()
        self.packed = packed  # keeps the borrowed buffer alive
        self.n = int(n)
        self.m, self.stride = packed.shape
        self.device = packed.device
        h = ctypes.c_void_p()
        if mu is not None:
            mu = mu.to(self.device, torch.float64).contiguous()
            scale = scale.to(self.device, torch.float64).contiguous()
        with torch.cuda.device(self.device):
            _check(lib().gkl_init(ctypes.byref(h), _ptr(packed), self.n, self.m, self.stride, _ptr(mu), _ptr(scale),
                                  _stream()))
        self._h = h
        self._weights = (None, None)
        # bumped by every solve and weight change: a backward pass checks that the
        # handle still holds the triplets its forward pass produced
        self.generation = 0
        self._last = (0, torch.float64)  # k and dtype of the last solve

    def close(self):
        if getattr(self, "_h", None):
            lib().gkl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        lib().gkl_set_stream(self._h, _stream())

    def set_weights(self, s: torch.Tensor | None = None, w: torch.Tensor | None = None):
        self._sync_stream()
        s = None if s is None else s.to(self.device, torch.float32).contiguous()
        w = None if w is None else w.to(self.device, torch.float32).contiguous()
        if s is not None:
            _need_buffer(s, (self.n,), what="sample weights s")
        if w is not None:
            _need_buffer(w, (self.m,), what="SNP weights w")
        self.generation += 1
        _check(lib().gkl_set_weights(self._h, _ptr(s), _ptr(w)), self._h)
        self._weights = (s, w)

    def matvec(self, v: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        prec = FP64 if v.dtype == torch.float64 else FP32
        assert v.is_cuda and v.dtype in (torch.float32, torch.float64) and v.numel() == self.m and v.is_contiguous()
        y = out if out is not None else torch.empty(self.n, dtype=v.dtype, device=self.device)
        _need_buffer(y, (self.n,), v.dtype, True, "out")
        self._sync_stream()
        _check(lib().gkl_matvec(self._h, prec, _ptr(v), _ptr(y)), self._h)
        return y

    def rmatvec(self, u: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        prec = FP64 if u.dtype == torch.float64 else FP32
        assert u.is_cuda and u.dtype in (torch.float32, torch.float64) and u.numel() == self.n and u.is_contiguous()
        x = out if out is not None else torch.empty(self.m, dtype=u.dtype, device=self.device)
        _need_buffer(x, (self.m,), u.dtype, True, "out")
        self._sync_stream()
        _check(lib().gkl_rmatvec(self._h, prec, _ptr(u), _ptr(x)), self._h)
        return x

    def matmat(self, X: torch.Tensor, transpose: bool = False, digits: int = 8,
               out: torch.Tensor | None = None) -> torch.Tensor:
        """Block product on the tensor cores: A X (X m x q) or A^T X (X n x q),
        q <= 32, FP32; `digits` 8 (finer than FP32) or 4 (16-bit fixed point).
        X and the result are row-major q x rows tensors (column-major rows x q)."""
        rows_in, rows_out = (self.n, self.m) if transpose else (self.m, self.n)
        assert X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.shape[1] == rows_in
        assert X.is_contiguous()
        q = X.shape[0]
        Y = out if out is not None else torch.empty((q, rows_out), dtype=torch.float32, device=self.device)
        _need_buffer(Y, (q, rows_out), torch.float32, True, "out")
        self._sync_stream()
        _check(lib().gkl_matmat(self._h, int(transpose), q, digits, _ptr(X), rows_in, _ptr(Y), rows_out), self._h)
        return Y

    def svd(self, k: int, ell: int, reorth: str = "dgks", precision: str = "fp64", tol: float = 1e-10,
            maxit: int = 1000, k_keep: int = 0, omega: float = 0.0, seed: int = 1,
            v0: torch.Tensor | None = None, want_u: bool = True, want_v: bool = True, profile: bool = False,
            U: torch.Tensor | None = None, V: torch.Tensor | None = None, raise_on_fail: bool = True,
            block: int = 0, out_host: bool = False) -> SVDResult:
        """Top-k triplets.  U and V come back as n x k and m x k views of
        column-major buffers, on the device, or in pinned host memory with
        out_host=True (the library copies them there).  Caller buffers U and
        V, if given, are contiguous k x n and k x m tensors of the solve's
        dtype (the column-major layout); v0 has m entries."""
        prec = _PREC[precision]
        dt = _DTYPE[prec]
        o = Opts()
        lib().gkl_opts_default(ctypes.byref(o))
        o.k, o.ell, o.k_keep, o.reorth, o.precision, o.maxit = k, ell, k_keep, _REORTH[reorth], prec, maxit
        o.tol, o.omega, o.seed, o.profile = tol, omega, seed, int(profile)
        o.block, o.out_host = block, int(out_host)
        if v0 is not None:
            v0 = v0.to(self.device, dt).contiguous()
            _need_buffer(v0, (self.m,), what="v0")
            o.v0 = v0.data_ptr()
        where = dict(device="cpu", pin_memory=True) if out_host else dict(device=self.device)
        if U is None and want_u:
            U = torch.empty((k, self.n), dtype=dt, **where)  # column-major n x k
        if V is None and want_v:
            V = torch.empty((k, self.m), dtype=dt, **where)
        if U is not None:
            _need_buffer(U, (k, self.n), dt, what="U")
        if V is not None:
            _need_buffer(V, (k, self.m), dt, what="V")
        sigma = np.zeros(k)
        resid = np.zeros(k)
        info = Info()
        self._sync_stream()
        self.generation += 1
        st = lib().gkl_svd(self._h, ctypes.byref(o), sigma.ctypes.data_as(ctypes.c_void_p), _ptr(U), _ptr(V),
                           resid.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info))
        if st not in (OK, NOT_CONVERGED, RANK_DEFICIENT) and raise_on_fail:
            _check(st, self._h)
        self._last = (k, dt)
        return SVDResult(sigma, None if U is None else U.T, None if V is None else V.T, resid, info.as_dict(), st)

    def scores(self, out_host: bool = False) -> torch.Tensor:
        """PC scores U diag(sigma) of the last successful solve (n x k view of a
        column-major buffer), computed by the library."""
        k = self._last_k()
        dt = self._last_dtype
        where = dict(device="cpu", pin_memory=True) if out_host else dict(device=self.device)
        S = torch.empty((k, self.n), dtype=dt, **where)
        self._sync_stream()
        _check(lib().gkl_scores(self._h, _ptr(S), int(out_host)), self._h)
        return S.T

    def sync(self):
        """Synchronise the handle's stream; raises if a tensor-core product's
        bounded wait ran out since the last check."""
        _check(lib().gkl_sync(self._h), self._h)

    def _last_k(self):
        return self._last[0]

    @property
    def _last_dtype(self):
        return self._last[1]

    def grad(self, sigma_bar=None, scores_bar: torch.Tensor | None = None, want_w: bool = True,
             want_s: bool = True, min_relgap: float = 1e-3, dtype=None):
        """(dL/ds, dL/dw) for the triplets of the last converged svd() call.

        sigma_bar: k adjoints of the singular values; scores_bar: n x k
        adjoints of the PC scores U diag(sigma).  dtype: the precision of that
        solve (float64 after "fp64", float32 otherwise; None = as it was)."""
        if dtype is None:
            dtype = self._last_dtype
        sb = None
        if sigma_bar is not None:
            sb = np.ascontiguousarray(np.asarray(sigma_bar, dtype=np.float64))
            if self._last_k() and sb.shape != (self._last_k(),):  # before any solve the library says ERR_STATE
                raise ValueError(f"sigma_bar: expected {self._last_k()} entries, got shape {sb.shape}")
        Sb = None
        if scores_bar is not None:
            if self._last_k() and tuple(scores_bar.shape) != (self.n, self._last_k()):
                raise ValueError(f"scores_bar: expected shape {(self.n, self._last_k())}, "
                                 f"got {tuple(scores_bar.shape)}")
            Sb = scores_bar.to(self.device, dtype).t().contiguous()  # column-major n x k
        gw = torch.empty(self.m, dtype=dtype, device=self.device) if want_w else None
        gs = torch.empty(self.n, dtype=dtype, device=self.device) if want_s else None
        self._sync_stream()
        _check(lib().gkl_grad(self._h, None if sb is None else sb.ctypes.data_as(ctypes.c_void_p), _ptr(Sb),
                              _ptr(gw), _ptr(gs), min_relgap), self._h)
        return gs, gw


class GKLFunction(torch.autograd.Function):
    """(s, w) -> (sigma, scores) with the gradient computed by gkl_grad.

    forward: sets the per-sample weights s (n) and per-SNP weights w (m) on
    the handle and runs the top-k solve; returns sigma (k, float64) and the PC
    scores U diag(sigma) (n x k).  backward: dL/ds and dL/dw from the adjoints
    of sigma and of the scores."""

    @staticmethod
    def forward(ctx, s, w, handle: GKL, solve_kw: dict, min_relgap: float):
        handle.set_weights(s.detach(), w.detach())
        r = handle.svd(**solve_kw)
        if not r.converged:
            raise GKLError(NOT_CONVERGED, "forward solve did not converge")
        ctx.handle, ctx.min_relgap = handle, min_relgap
        ctx.generation = handle.generation
        ctx.dtype = r.U.dtype
        ctx.sdtype, ctx.wdtype = s.dtype, w.dtype
        sigma = torch.tensor(r.sigma, dtype=torch.float64, device=r.U.device)
        scores = handle.scores()
        return sigma, scores

    @staticmethod
    def backward(ctx, sigma_bar, scores_bar):
        if ctx.handle.generation != ctx.generation:
            raise GKLError(ERR_STATE, "the handle was solved again or its weights changed after this forward pass; "
                                      "its stored triplets no longer belong to this graph")
        sb = None if sigma_bar is None else sigma_bar.detach().double().cpu().numpy()
        gs, gw = ctx.handle.grad(sb, scores_bar, min_relgap=ctx.min_relgap, dtype=ctx.dtype)
        return gs.to(ctx.sdtype), gw.to(ctx.wdtype), None, None, None
