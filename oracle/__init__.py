"""CPU oracle for the genotype PCA path -- TEST INFRASTRUCTURE ONLY.

Plain FP64 restatement of what the GPU library computes (``oracle.c``, plus the
Marchenko-Pastur law in ``mp.py`` and the gradient formulas in ``grad.py``).
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library.

Citations are to arXiv:1808.03374 (Chen, Noack, Edelman): section 3 for
Golub-Kahan-Lanczos bidiagonalisation with thick restart, CGS2 full
reorthogonalisation and the residual convergence test; Table 3 for the
||Delta theta||_1 error measure; section 2, Eqs. 4-5 for the Marchenko-Pastur
law.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, FP contraction off so every product and sum is
    rounded exactly as written)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "liboracle.so")
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


class _Mat(ctypes.Structure):
    _fields_ = [("packed", ctypes.c_void_p), ("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("stride", ctypes.c_int64), ("mu", ctypes.c_void_p), ("d", ctypes.c_void_p),
                ("s", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("ell", ctypes.c_int32), ("k_keep", ctypes.c_int32),
                ("maxit", ctypes.c_int32), ("tol", ctypes.c_double), ("seed", ctypes.c_uint64)]


class _Info(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int64), ("restarts", ctypes.c_int32), ("breakdowns", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("cycles", ctypes.c_int32),
                ("max_rel_resid", ctypes.c_double), ("dtheta1", ctypes.c_double)]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            vp, i64 = ctypes.c_void_p, ctypes.c_int64
            P = ctypes.POINTER
            lib.orc_colstats.argtypes = [vp, i64, i64, i64, vp, vp, vp]
            lib.orc_unpack.argtypes = [P(_Mat), vp]
            lib.orc_matvec.argtypes = [P(_Mat), vp, vp]
            lib.orc_rmatvec.argtypes = [P(_Mat), vp, vp]
            lib.orc_matvec_rows.argtypes = [P(_Mat), vp, vp, i64, vp]
            lib.orc_rmatvec_cols.argtypes = [P(_Mat), vp, vp, i64, vp]
            lib.orc_matmat.argtypes = [P(_Mat), vp, i64, vp]
            lib.orc_rmatmat.argtypes = [P(_Mat), vp, i64, vp]
            lib.orc_jacobi_svd.argtypes = [i64, i64, vp, vp, vp, vp]
            lib.orc_jacobi_svd.restype = ctypes.c_int
            lib.orc_gkl.argtypes = [P(_Mat), P(_Opts), vp, vp, vp, vp, vp, P(_Info), vp, vp, vp]
            lib.orc_gkl.restype = ctypes.c_int
            lib.orc_sign_fix.argtypes = [i64, i64, i64, vp, vp]
            _LIB = lib
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Matrix:
    """A = diag(s) (G - 1 mu^T)[observed] diag(d * w), G given 2-bit packed."""
    packed: np.ndarray
    n: int
    mu: np.ndarray
    d: np.ndarray
    s: np.ndarray | None = None
    w: np.ndarray | None = None

    def __post_init__(self):
        self.packed = np.ascontiguousarray(self.packed, dtype=np.uint8)
        self.mu, self.d, self.s, self.w = _f64(self.mu), _f64(self.d), _f64(self.s), _f64(self.w)

    @property
    def m(self):
        return self.packed.shape[0]

    @property
    def stride(self):
        return self.packed.shape[1]

    def _c(self):
        c = _Mat()
        c.packed, c.n, c.m, c.stride = self.packed.ctypes.data, self.n, self.m, self.stride
        c.mu, c.d, c.s, c.w = _ptr(self.mu), _ptr(self.d), _ptr(self.s), _ptr(self.w)
        return c

    @classmethod
    def from_packed(cls, packed, n, s=None, w=None):
        mu, d, _ = colstats(packed, n)
        return cls(packed, n, mu, d, s, w)

    def dense(self) -> np.ndarray:
        A = np.empty((self.m, self.n), dtype=np.float64)  # column-major n x m == row-major m x n
        _lib().orc_unpack(ctypes.byref(self._c()), A.ctypes.data)
        return A.T

    def matvec(self, v):
        v = _f64(v)
        y = np.empty(self.n)
        _lib().orc_matvec(ctypes.byref(self._c()), v.ctypes.data, y.ctypes.data)
        return y

    def rmatvec(self, u):
        u = _f64(u)
        x = np.empty(self.m)
        _lib().orc_rmatvec(ctypes.byref(self._c()), u.ctypes.data, x.ctypes.data)
        return x

    def matmat(self, X):
        """A X for an m x k matrix X (each column as matvec computes it)."""
        X = np.asfortranarray(X, dtype=np.float64)
        k = X.shape[1]
        Y = np.empty((self.n, k), order="F")
        _lib().orc_matmat(ctypes.byref(self._c()), X.ctypes.data, k, Y.ctypes.data)
        return Y

    def rmatmat(self, U):
        """A^T U for an n x k matrix U (each column as rmatvec computes it)."""
        U = np.asfortranarray(U, dtype=np.float64)
        k = U.shape[1]
        X = np.empty((self.m, k), order="F")
        _lib().orc_rmatmat(ctypes.byref(self._c()), U.ctypes.data, k, X.ctypes.data)
        return X

    def matvec_rows(self, v, rows):
        v, rows = _f64(v), np.ascontiguousarray(rows, dtype=np.int64)
        y = np.empty(len(rows))
        _lib().orc_matvec_rows(ctypes.byref(self._c()), v.ctypes.data, rows.ctypes.data, len(rows), y.ctypes.data)
        return y

    def rmatvec_cols(self, u, cols):
        u, cols = _f64(u), np.ascontiguousarray(cols, dtype=np.int64)
        x = np.empty(len(cols))
        _lib().orc_rmatvec_cols(ctypes.byref(self._c()), u.ctypes.data, cols.ctypes.data, len(cols), x.ctypes.data)
        return x


def colstats(packed, n):
    """Per-SNP mean, inverse population SD (0 if monomorphic) and observed count."""
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    m, stride = packed.shape
    mu, d, nobs = np.empty(m), np.empty(m), np.empty(m, dtype=np.int64)
    _lib().orc_colstats(packed.ctypes.data, n, m, stride, mu.ctypes.data, d.ctypes.data, nobs.ctypes.data)
    return mu, d, nobs


def jacobi_svd(A):
    """One-sided Jacobi SVD of a tall matrix: returns U, sigma (descending), V, sweeps."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    r, c = A.shape
    assert r >= c
    sig, U, V = np.empty(c), np.empty((r, c), order="F"), np.empty((c, c), order="F")
    sweeps = _lib().orc_jacobi_svd(r, c, A.ctypes.data, sig.ctypes.data, U.ctypes.data, V.ctypes.data)
    return U, sig, V, sweeps


def sign_fix(U, V):
    """Make the largest-|.| entry of each V column positive (first on ties), flipping U along."""
    U = np.array(U, dtype=np.float64, order="F", copy=True)
    V = np.array(V, dtype=np.float64, order="F", copy=True)
    _lib().orc_sign_fix(U.shape[0], V.shape[0], V.shape[1], U.ctypes.data, V.ctypes.data)
    return U, V


@dataclass
class GKLResult:
    sigma: np.ndarray
    U: np.ndarray
    V: np.ndarray
    resid: np.ndarray
    status: int
    pairs: int
    restarts: int
    breakdowns: int
    converged: bool
    cycles: int
    max_rel_resid: float
    dtheta1: float
    Ub: np.ndarray | None = None
    Vb: np.ndarray | None = None
    B: np.ndarray | None = None


def gkl(M: Matrix, k: int, ell: int, tol: float, v0, maxit: int = 200, k_keep: int = 0,
        seed: int = 0, bases: bool = False) -> GKLResult:
    """Thick-restarted GKL with CGS2 full reorthogonalisation (section 3)."""
    o = _Opts()
    o.k, o.ell, o.k_keep, o.maxit, o.tol, o.seed = k, ell, k_keep, maxit, tol, seed
    v0 = _f64(v0)
    sig, resid = np.empty(k), np.empty(k)
    U, V = np.empty((M.n, k), order="F"), np.empty((M.m, k), order="F")
    Ub = np.empty((M.n, ell), order="F") if bases else None
    Vb = np.empty((M.m, ell + 1), order="F") if bases else None
    B = np.empty((ell, ell), order="F") if bases else None
    info = _Info()
    st = _lib().orc_gkl(ctypes.byref(M._c()), ctypes.byref(o), v0.ctypes.data, sig.ctypes.data, U.ctypes.data,
                        V.ctypes.data, resid.ctypes.data, ctypes.byref(info), _ptr(Ub), _ptr(Vb), _ptr(B))
    if st < 0:
        raise ValueError("orc_gkl: bad arguments")
    return GKLResult(sig, U, V, resid, st, info.pairs, info.restarts, info.breakdowns, bool(info.converged),
                     info.cycles, info.max_rel_resid, info.dtheta1, Ub, Vb, B)
