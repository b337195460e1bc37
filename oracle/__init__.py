"""CPU FP64 oracle for the SPD solve path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The product (the CUDA library and its
binding in ``paper_2601_14466_gb300``) never imports it and shares no code with
it.

The arithmetic lives in ``oracle.c`` (plain C, no BLAS); this module builds it
with gcc and exposes each routine through ctypes on NumPy arrays.  Matrices are
column-major (``numpy.asfortranarray``); only the lower triangle of a
symmetric ``A`` is read.  Paper: "Software design", the ``potrs`` workflow
(SPD solve by Cholesky, optional log det).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_default = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int
_GCC = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
        "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no fused multiply-add)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.run(_GCC + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _f64(a) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    return np.asfortranarray(a)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _ld(a: np.ndarray) -> int:
    return max(1, a.shape[0])


class Oracle:
    """ctypes front end over one compiled copy of oracle.c."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        lib.oracle_potrf.argtypes = [_I, _D, _I]
        lib.oracle_potrf.restype = _I
        lib.oracle_potrs.argtypes = [_I, _I, _D, _I, _D, _I]
        lib.oracle_potrs.restype = None
        lib.oracle_posv.argtypes = [_I, _I, _D, _I, _D, _I]
        lib.oracle_posv.restype = _I
        lib.oracle_resid_dot2.argtypes = [_I, _I, _D, _I, _D, _I, _D, _I, _D, _I]
        lib.oracle_resid_dot2.restype = None
        lib.oracle_norm_inf.argtypes = [_I, _D, _I]
        lib.oracle_norm_inf.restype = ctypes.c_double
        lib.oracle_bwd_err.argtypes = [_I, _I, _D, _I, _D, _I, _D, _I, _D]
        lib.oracle_bwd_err.restype = ctypes.c_double
        lib.oracle_bwd_err_rows.argtypes = [_I, _I, _D, _I, _D, _I, _D, _I, _D]
        lib.oracle_bwd_err_rows.restype = ctypes.c_double
        lib.oracle_rowmajor_to_colmajor.argtypes = [ctypes.c_longlong, ctypes.c_longlong, _D, _D]
        lib.oracle_rowmajor_to_colmajor.restype = None
        lib.oracle_logdet.argtypes = [_I, _D, _I]
        lib.oracle_logdet.restype = ctypes.c_double
        lib.oracle_grad.argtypes = [_I, _I, _D, _I, _D, _I, _D, _I, _D, _D, _D, _I]
        lib.oracle_grad.restype = _I
        lib.oracle_ge_solve.argtypes = [_I, _I, _D, _I, _D, _I]
        lib.oracle_ge_solve.restype = _I
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = _I
        lib.oracle_set_threads.argtypes = [_I]
        lib.oracle_set_threads.restype = None
        self.lib = lib
        self.path = path

    def threads(self) -> int:
        return self.lib.oracle_num_threads()

    def set_threads(self, t: int) -> None:
        self.lib.oracle_set_threads(int(t))

    def potrf(self, A):
        """Lower Cholesky factor of the symmetric matrix held in lower(A).

        Returns ``(L, info)``: ``L`` is a new column-major array whose lower
        triangle holds the factor (the upper triangle is copied through
        untouched, as the routine never references it); ``info`` is 0 or the
        1-based column of the first pivot that is not positive."""
        L = _f64(A).copy(order="F")
        info = self.lib.oracle_potrf(L.shape[0], _p(L), _ld(L))
        return L, int(info)

    def potrs(self, L, B):
        """Solve (L L^T) X = B with the lower factor in lower(L)."""
        L = _f64(L)
        X = _f64(B).copy(order="F")
        self.lib.oracle_potrs(L.shape[0], X.shape[1], _p(L), _ld(L), _p(X), _ld(X))
        return X

    def posv(self, A, B):
        """Cholesky solve of A X = B (lower(A) read); returns ``(X, info)``."""
        A2 = _f64(A).copy(order="F")
        X = _f64(B).copy(order="F")
        info = self.lib.oracle_posv(A2.shape[0], X.shape[1], _p(A2), _ld(A2), _p(X), _ld(X))
        return X, int(info)

    def resid_dot2(self, A, X, B):
        """R = B - A X (A symmetric, lower read), each entry by compensated Dot2."""
        A, X, B = _f64(A), _f64(X), _f64(B)
        n, nrhs = X.shape
        R = np.zeros((n, nrhs), order="F")
        self.lib.oracle_resid_dot2(n, nrhs, _p(A), _ld(A), _p(X), _ld(X), _p(B), _ld(B),
                                   _p(R), _ld(R))
        return R

    def norm_inf(self, A) -> float:
        A = _f64(A)
        return float(self.lib.oracle_norm_inf(A.shape[0], _p(A), _ld(A)))

    def bwd_err(self, A, X, B):
        """Normwise backward error per column and its maximum:
        eta_j = ||b_j - A x_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf)."""
        A, X, B = _f64(A), _f64(X), _f64(B)
        n, nrhs = X.shape
        eta = np.zeros(nrhs)
        worst = self.lib.oracle_bwd_err(n, nrhs, _p(A), _ld(A), _p(X), _ld(X), _p(B), _ld(B),
                                        _p(eta))
        return float(worst), eta

    def bwd_err_rows(self, A, X, B):
        """oracle_bwd_err's numbers, bit for bit, with A read once (for matrices
        of tens of GB).  A, X and B may be any column-major float64 arrays
        (A: only its lower triangle is read)."""
        A, X, B = _f64(A), _f64(X), _f64(B)
        n, nrhs = X.shape
        eta = np.zeros(nrhs)
        worst = self.lib.oracle_bwd_err_rows(n, nrhs, _p(A), _ld(A), _p(X), _ld(X), _p(B),
                                             _ld(B), _p(eta))
        return float(worst), eta

    def rowmajor_to_colmajor(self, buf, m, n):
        """The m*n buffer holding an m x n matrix row-major, rewritten in
        column-major order (a new flat float64 array)."""
        src = np.ascontiguousarray(np.asarray(buf, dtype=np.float64).reshape(-1))
        assert src.size == m * n
        out = np.empty(m * n)
        self.lib.oracle_rowmajor_to_colmajor(m, n, _p(src), _p(out))
        return out

    def logdet(self, L) -> float:
        """log det A = 2 sum log L_ii from a lower Cholesky factor."""
        L = _f64(L)
        return float(self.lib.oracle_logdet(L.shape[0], _p(L), _ld(L)))

    def grad(self, A, B, Xbar):
        """Adjoint of X = A^{-1} B.  Returns ``(X, Bbar, Abar, info)`` with
        Bbar = A^{-1} Xbar and Abar = -(Bbar X^T + X Bbar^T)/2 (full symmetric)."""
        A, B, Xbar = _f64(A), _f64(B), _f64(Xbar)
        n, nrhs = B.shape
        X = np.zeros((n, nrhs), order="F")
        Bbar = np.zeros((n, nrhs), order="F")
        Abar = np.zeros((n, n), order="F")
        info = self.lib.oracle_grad(n, nrhs, _p(A), _ld(A), _p(B), _ld(B), _p(Xbar), _ld(Xbar),
                                    _p(X), _p(Bbar), _p(Abar), _ld(Abar))
        return X, Bbar, Abar, int(info)

    def ge_solve(self, A, B):
        """Gaussian elimination with partial pivoting on the symmetric matrix held
        in lower(A) (tiny n only).  Returns ``(X, info)``."""
        A = _f64(A)
        X = _f64(B).copy(order="F")
        info = self.lib.oracle_ge_solve(A.shape[0], X.shape[1], _p(A), _ld(A), _p(X), _ld(X))
        return X, int(info)


def default() -> Oracle:
    """The oracle built from oracle.c as committed."""
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def variant(source: str, workdir: str) -> Oracle:
    """Compile an edited copy of oracle.c (``source`` is its full text) into
    ``workdir`` and load it.  Tests use this to plant a mistake in the oracle
    and check that the pins catch it."""
    src = os.path.join(workdir, "oracle_variant.c")
    lib = os.path.join(workdir, "liboracle_variant.so")
    with open(src, "w") as f:
        f.write(source)
    subprocess.run(_GCC + [src, "-o", lib, "-lm"], check=True)
    return Oracle(lib)


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def threads() -> int:
    return default().threads()


def set_threads(t: int) -> None:
    default().set_threads(t)


def potrf(A):
    return default().potrf(A)


def potrs(L, B):
    return default().potrs(L, B)


def posv(A, B):
    return default().posv(A, B)


def resid_dot2(A, X, B):
    return default().resid_dot2(A, X, B)


def norm_inf(A) -> float:
    return default().norm_inf(A)


def bwd_err(A, X, B):
    return default().bwd_err(A, X, B)


def bwd_err_rows(A, X, B):
    return default().bwd_err_rows(A, X, B)


def rowmajor_to_colmajor(buf, m, n):
    return default().rowmajor_to_colmajor(buf, m, n)


def logdet(L) -> float:
    return default().logdet(L)


def grad(A, B, Xbar):
    return default().grad(A, B, Xbar)


def ge_solve(A, B):
    return default().ge_solve(A, B)
