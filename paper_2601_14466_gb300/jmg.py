"""Python binding of libjmg.so (ctypes): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; PyTorch supplies
device memory and the stream.  There is no CPU fallback: if the library is
missing or no CUDA device is present, the calls raise.

Raw entry points keep the C names (``jmg_potrf``, ``jmg_potrs``, ``jmg_posv``,
``jmg_workspace_size``, ``jmg_logdet``, ...) and take integers / pointers.  The
tensor-level helpers (``potrf_``, ``potrs_``, ``posv``, ``logdet``) take torch
tensors in column-major layout (``stride(0) == 1``): for a symmetric matrix held
row-major, ``A.mT`` is such a view of the same storage.

Paper: "Software design" -- potrs = Cholesky potrf + potrs (optional log det).
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

from . import _build

_lock = threading.Lock()
_lib = None

JMG_F64, JMG_F32 = 0, 1
PREC = {"fp64": 0, "native": 0, "bf16": 1, "fp16": 2, "fp8": 3, "fp32": 4}
REFINE = {"ir": 0, "pcg": 1, "auto": 2}
OP_POTRF, OP_POTRS, OP_POSV, OP_POSV_HOST = 0, 1, 2, 3

STATUS = {0: "ok", 1: "CUDA error", 2: "workspace too small", 3: "matrix is not positive definite",
          4: "refinement did not reach the tolerance", 5: "device-side wait timed out",
          6: "unsupported option combination", 7: "alignment requirement not met"}


class JmgError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        msg = STATUS.get(status, "illegal argument %d" % -status if status < 0 else "status %d" % status)
        super().__init__("%s: %s (status %d)" % (where or "jmg", msg, status))


class Options(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("NB", ctypes.c_int), ("prec", ctypes.c_int),
                ("words", ctypes.c_int), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("refine", ctypes.c_int), ("shift_retry", ctypes.c_int), ("timing", ctypes.c_int),
                ("reuse_factor", ctypes.c_int), ("resid", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("info", ctypes.c_int), ("iters", ctypes.c_int),
                ("refine_used", ctypes.c_int), ("words_used", ctypes.c_int),
                ("factor_tries", ctypes.c_int), ("bwd_err", ctypes.c_double),
                ("shift", ctypes.c_double), ("anorm", ctypes.c_double),
                ("t_factor_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("t_refine_ms", ctypes.c_double), ("t_resid_gpu_ms", ctypes.c_double),
                ("n_resid", ctypes.c_int), ("n_hist", ctypes.c_int),
                ("eta_hist", ctypes.c_double * 32), ("t_solve_gpu_ms", ctypes.c_double),
                ("n_solve", ctypes.c_int), ("t_factor_gpu_ms", ctypes.c_double),
                ("h2d_bytes", ctypes.c_longlong), ("d2h_bytes", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I = ctypes.c_int
_SZ = ctypes.c_size_t

_SIGS = {
    "jmg_default_options": (None, [ctypes.POINTER(Options)]),
    "jmg_workspace_size": (_SZ, [_I, _I, _I, _I, ctypes.POINTER(Options)]),
    "jmg_potrf": (_I, [_I, _P, _I, _I, _P, ctypes.POINTER(Options), _P, _SZ, _P]),
    "jmg_potrs": (_I, [_I, _I, _P, _I, _P, _I, _I, _P, _SZ, _P]),
    "jmg_potrs_static": (_I, [_I, _I, _P, _I, _P, _I, _I, _P]),
    "jmg_posv": (_I, [_I, _I, _P, _I, _P, _I, _I, _P, ctypes.POINTER(Options),
                      ctypes.POINTER(Stats), _P, _SZ, _P]),
    "jmg_posv_host": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _I, ctypes.POINTER(_I),
                           ctypes.POINTER(Options), ctypes.POINTER(Stats), _P, _SZ, _P]),
    "jmg_logdet": (_I, [_I, _P, _I, _I, _P, _P]),
    "jmg_status_string": (ctypes.c_char_p, [_I]),
    "jmg_sym_grad": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P]),
    "jmg_dev_syrk_tc": (_I, [_I, _I, _I, _P, _P, _I, _I, _P, _I, _P, _P]),
    "jmg_dev_syrk_fp8": (_I, [_I, _I, _I, _P, _I, _P, _P, _I, _P, _P]),
    "jmg_dev_syrk_fp8_chunks": (_I, [_I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _P]),
    "jmg_dev_residual_workspace": (_SZ, [_I, _I]),
    "jmg_dev_residual": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _P, _SZ, _P]),
    "jmg_dev_residual_split_workspace": (_SZ, [_I, _I]),
    "jmg_dev_residual_split": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _P, _P, _SZ, _P]),
    "jmg_dev_norm_inf": (_I, [_I, _P, _I, _P, _P, _SZ, _P]),
    "jmg_dev_probe": (_I, [_I, _I, _I, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "jmg_dev_launch_count": (ctypes.c_longlong, []),
    "jmg_dev_set_wait_limit_ns": (ctypes.c_ulonglong, [ctypes.c_ulonglong]),
    "jmg_dev_trsv_leaderless": (_I, [_I, _I, _P, _I, _P, _I, _I, _P, _P, _P]),
    "jmg_dev_syrk_tc_idle_producer": (_I, [_I, _I, _I, _P, _P, _I, _I, _P, _I, _P, _P]),
    "jmg_dev_quant_fp8": (_I, [_I, _I, _P, _I, _P, _I, _P, _P]),
    "jmg_dev_sv_workspace": (_SZ, [_I, _I]),
    "jmg_dev_sv_potrs": (_I, [_I, _I, _P, _I, _P, _I, _P, _SZ, _P]),
    "jmg_potrs_static_status": (_I, [ctypes.POINTER(_I), _P]),
    "jmg_posv_batched": (_I, [_I, _I, _I, _P, _I, ctypes.c_longlong, _P, _I, ctypes.c_longlong, _I,
                              _P, _P]),
    "jmg_layout_workspace": (_SZ, [ctypes.c_longlong, ctypes.c_longlong, _I]),
    "jmg_rowmajor_to_colmajor": (_I, [ctypes.c_longlong, ctypes.c_longlong, _P, _I, _P, _SZ, _P]),
    "jmg_colmajor_to_rowmajor": (_I, [ctypes.c_longlong, ctypes.c_longlong, _P, _I, _P, _SZ, _P]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libjmg.so (building it first if it is missing and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB) or (build_if_missing and not _build.up_to_date()):
                if not build_if_missing:
                    raise RuntimeError("libjmg.so is not built: run __graft_entry__.build()")
                _build.build()
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def _chk(st: int, where: str):
    if st != 0:
        raise JmgError(st, where)


def _stream(dev) -> int:
    return torch.cuda.current_stream(dev).cuda_stream


def _need_cuda(*ts):
    for t in ts:
        if not t.is_cuda:
            raise ValueError("jmg: tensors must live on a CUDA device (no CPU path)")


def _colmajor(t: torch.Tensor, name: str):
    if t.dim() != 2:
        raise ValueError("%s must be 2-D" % name)
    n, m = t.shape
    if t.stride(0) != 1 and not (m == 1 and t.is_contiguous()):
        raise ValueError("%s must be column-major (stride(0) == 1); for a symmetric row-major "
                         "matrix pass its .mT view" % name)
    ld = t.stride(1) if m > 1 else max(n, 1)
    return t.data_ptr(), max(ld, max(n, 1))


def colmajor_copy(t: torch.Tensor) -> torch.Tensor:
    """A NEW column-major copy of a 2-D tensor (stride (1, rows)); never an alias."""
    if t.dim() != 2:
        t = t.reshape(-1, 1)
    out = torch.empty((t.shape[1], t.shape[0]), dtype=t.dtype, device=t.device).t()
    out.copy_(t)
    return out


def default_options(**kw) -> Options:
    o = Options()
    load().jmg_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "prec" and isinstance(v, str):
            v = PREC[v]
        if k == "refine" and isinstance(v, str):
            v = REFINE[v]
        setattr(o, k, v)
    return o


def workspace_size(op: int, n: int, nrhs: int, opts: Options | None = None,
                   dtype: int = JMG_F64) -> int:
    return int(load().jmg_workspace_size(op, n, nrhs, dtype, ctypes.byref(opts) if opts else None))


def workspace(op: int, n: int, nrhs: int, opts: Options | None, device,
              dtype: int = JMG_F64) -> torch.Tensor:
    nbytes = workspace_size(op, n, nrhs, opts, dtype)
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


# ------------------------------------------------------------------ tensor helpers


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return JMG_F64
    if t.dtype == torch.float32:
        return JMG_F32
    raise TypeError("float64 or float32 storage only, got %s" % t.dtype)


def potrf_(A: torch.Tensor, *, nb: int = 128, info: torch.Tensor | None = None) -> torch.Tensor:
    """Cholesky factorisation in place: lower(A) <- L (FP64 or FP32, column-major).
    Returns the device info tensor (int32, 1 element); asynchronous."""
    _need_cuda(A)
    dt = _dtype_code(A)
    p, lda = _colmajor(A, "A")
    n = A.shape[0]
    if info is None:
        info = torch.zeros(1, dtype=torch.int32, device=A.device)
    o = default_options(nb=nb)
    st = load().jmg_potrf(n, p, lda, dt, info.data_ptr(), ctypes.byref(o), None, 0,
                          _stream(A.device))
    _chk(st, "jmg_potrf")
    return info


def potrs_(L: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """Solve (L L^T) X = B in place on B (column-major); asynchronous."""
    _need_cuda(L, B)
    dt = _dtype_code(L)
    if B.dtype != L.dtype:
        raise TypeError("potrs_: L and B must have the same dtype")
    pl, lda = _colmajor(L, "L")
    pb, ldb = _colmajor(B, "B")
    work = workspace(OP_POTRS, L.shape[0], B.shape[1], None, L.device)
    st = load().jmg_potrs(L.shape[0], B.shape[1], pl, lda, pb, ldb, dt, work.data_ptr(),
                          work.numel(), _stream(L.device))
    _chk(st, "jmg_potrs")
    return B


@dataclass
class SolveInfo:
    status: int
    info: int
    iters: int
    bwd_err: float
    shift: float
    words: int
    factor_tries: int
    anorm: float
    t_factor_ms: float
    t_solve_ms: float
    t_refine_ms: float
    refine_used: int
    t_resid_gpu_ms: float = 0.0
    n_resid: int = 0
    eta_hist: tuple = ()
    t_solve_gpu_ms: float = 0.0
    n_solve: int = 0
    t_factor_gpu_ms: float = 0.0
    h2d_bytes: int = 0
    d2h_bytes: int = 0


def _solve_info(stats: Stats) -> SolveInfo:
    return SolveInfo(stats.status, stats.info, stats.iters, stats.bwd_err, stats.shift,
                     stats.words_used, stats.factor_tries, stats.anorm, stats.t_factor_ms,
                     stats.t_solve_ms, stats.t_refine_ms, stats.refine_used,
                     stats.t_resid_gpu_ms, stats.n_resid,
                     tuple(stats.eta_hist[i] for i in range(min(stats.n_hist, 32))),
                     stats.t_solve_gpu_ms, stats.n_solve, stats.t_factor_gpu_ms,
                     stats.h2d_bytes, stats.d2h_bytes)


def _options(prec, words, nb, tol, maxit, refine, shift_retry, timing, reuse_factor, resid,
             NB=None):
    return default_options(nb=nb, NB=NB, prec=prec, words=words, tol=tol, maxit=maxit, refine=refine,
                           shift_retry=int(shift_retry), timing=int(timing),
                           reuse_factor=int(reuse_factor),
                           resid={"auto": 0, "fp64": 1, "split": 2}[resid])


def posv(A: torch.Tensor, B: torch.Tensor, *, prec: str = "fp64", words: int = 1, nb: int = 128,
         tol: float = 1e-13, maxit: int = 300, refine: str = "auto", shift_retry: bool = True,
         overwrite_a: bool = False, work: torch.Tensor | None = None, check: bool = True,
         timing: bool = False, reuse_factor: bool = False, resid: str = "auto",
         NB: int | None = None):
    """Solve A X = B for SPD A (lower triangle of the column-major A read).

    prec "fp64": potrf + potrs in FP64 (A is overwritten with L only when
    ``overwrite_a``; otherwise a copy is factored).  prec "bf16"/"fp16": mixed
    precision with tensor-core trailing updates and FP64 refinement; A is
    preserved.  prec "fp32" (n <= 2048, nrhs <= 64): FP32 factor and FP64
    refinement in one persistent kernel with the stopping rule on the device.
    Returns ``(X, SolveInfo)``; X is a new column-major tensor."""
    _need_cuda(A, B)
    if A.dtype != B.dtype or A.dtype not in (torch.float64, torch.float32):
        raise TypeError("posv: A and B must both be float64 (any mode) or both float32 "
                        "(prec='fp64', i.e. the plain path in the storage type)")
    dt = _dtype_code(A)
    if dt == JMG_F32 and prec != "fp64":
        raise TypeError("posv: the mixed modes refine FP64 data; float32 takes prec='fp64'")
    squeeze = B.dim() == 1
    if squeeze:
        B = B.reshape(-1, 1)
    n, nrhs = A.shape[0], B.shape[1]
    X = colmajor_copy(B)
    o = _options(prec, words, nb, tol, maxit, refine, shift_retry, timing, reuse_factor, resid,
                 NB)
    Aw = A if (overwrite_a or o.prec != 0) else colmajor_copy(A)
    pa, lda = _colmajor(Aw, "A")
    px, ldx = _colmajor(X, "B")
    # the plain path reports through info (zeroed here); the mixed paths write it
    # themselves and report through the status and stats
    info = (torch.zeros if o.prec == 0 else torch.empty)(1, dtype=torch.int32, device=A.device)
    stats = Stats()
    if work is None:
        work = workspace(OP_POSV, n, nrhs, o, A.device)
    wp, wl = (work.data_ptr(), work.numel()) if work is not None else (None, 0)
    st = load().jmg_posv(n, nrhs, pa, lda, px, ldx, dt, info.data_ptr(), ctypes.byref(o),
                         ctypes.byref(stats), wp, wl, _stream(A.device))
    if o.prec == 0:
        info_h = int(info.item()) if check else 0
        si = SolveInfo(st, info_h, 0, float("nan"), 0.0, 0, 1, float("nan"), 0, 0, 0, -1)
        if check and (st != 0 or info_h != 0):
            raise JmgError(st if st else 3, "jmg_posv(info=%d)" % info_h)
    else:
        si = _solve_info(stats)
        if check and st != 0:
            raise JmgError(st, "jmg_posv")
    return (X[:, 0] if squeeze else X), si


def posv_host(A: torch.Tensor, B: torch.Tensor, *, prec: str = "fp64", words: int = 1,
              nb: int = 128, tol: float = 1e-13, maxit: int = 300, refine: str = "auto",
              shift_retry: bool = True, out: torch.Tensor | None = None,
              work: torch.Tensor | None = None, check: bool = True, timing: bool = False,
              reuse_factor: bool = False, resid: str = "auto", device=None):
    """Solve A X = B with A and B in HOST memory (CPU tensors, column-major;
    page-locked ones copy fastest) through ``jmg_posv_host``: A and B go
    to the GPU, the solve runs there in the library's kernels (modes as
    :func:`posv`), and X comes back.  Returns ``(X, SolveInfo)``: X is ``out``
    when given (a column-major CPU tensor, which may be B itself), else a new
    one; ``work`` is a device byte tensor of at least
    ``workspace_size(OP_POSV_HOST, ...)`` bytes.  Blocks until X is on the host."""
    if not torch.cuda.is_available():
        raise RuntimeError("jmg.posv_host: no CUDA device (the solve has no CPU path)")
    for t, name in ((A, "A"), (B, "B")):
        if t.is_cuda:
            raise ValueError("posv_host: %s must be a host (CPU) tensor; use posv for device data"
                             % name)
    if A.dtype != B.dtype:
        raise TypeError("posv_host: A and B must have the same dtype")
    dt = _dtype_code(A)
    if dt == JMG_F32 and prec != "fp64":
        raise TypeError("posv_host: the mixed modes refine FP64 data; float32 takes prec='fp64'")
    squeeze = B.dim() == 1
    if squeeze:
        B = B.reshape(-1, 1)
    if A.dim() != 2 or A.shape[0] != A.shape[1] or B.dim() != 2 or B.shape[0] != A.shape[0]:
        raise ValueError("posv_host: A (n, n) and B (n, nrhs) or (n,)")
    n, nrhs = A.shape[0], B.shape[1]
    if out is None:
        X = torch.empty((nrhs, n), dtype=B.dtype, pin_memory=B.is_pinned()).t()
    else:
        X = out.reshape(-1, 1) if out.dim() == 1 else out
        if X.is_cuda or X.dtype != B.dtype or tuple(X.shape) != (n, nrhs):
            raise ValueError("posv_host: out must be a host tensor shaped and typed like B")
    pa, lda = _colmajor(A, "A")
    pb, ldb = _colmajor(B, "B")
    px, ldx = _colmajor(X, "out")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None \
        else torch.device(device)
    o = _options(prec, words, nb, tol, maxit, refine, shift_retry, timing, reuse_factor, resid)
    if work is None:
        work = workspace(OP_POSV_HOST, n, nrhs, o, dev, dt)
    info = ctypes.c_int(0)
    stats = Stats()
    with torch.cuda.device(dev):
        st = load().jmg_posv_host(n, nrhs, pa, lda, pb, ldb, px, ldx, dt, ctypes.byref(info),
                                  ctypes.byref(o), ctypes.byref(stats), work.data_ptr(),
                                  work.numel(), _stream(dev))
    si = _solve_info(stats)
    si.status, si.info = st, info.value
    if check and st != 0:
        raise JmgError(st, "jmg_posv_host(info=%d)" % info.value)
    return (X[:, 0] if squeeze else X), si


def posv_batched(A: torch.Tensor, B: torch.Tensor):
    """Solve many small SPD systems at once: A (batch, n, n), symmetric (its
    row- and column-major forms coincide; the lower triangle is read), B
    (batch, n, nrhs); FP64 or FP32, n <= 128.  Returns ``(X, L, info)``: X
    (batch, n, nrhs) new, L the factors (a new (batch, n, n) tensor whose
    transpose per system holds L in its lower triangle), info (batch,) int32;
    asynchronous."""
    _need_cuda(A, B)
    if A.dim() != 3 or B.dim() != 3 or A.shape[0] != B.shape[0] or A.shape[1] != A.shape[2] \
            or B.shape[1] != A.shape[1]:
        raise ValueError("posv_batched: A (batch, n, n) and B (batch, n, nrhs)")
    if A.dtype != B.dtype:
        raise TypeError("posv_batched: A and B must have the same dtype")
    dt = _dtype_code(A)
    batch, n, nrhs = A.shape[0], A.shape[1], B.shape[2]
    Lw = A.transpose(1, 2).contiguous()        # per system: column-major copy of A
    Xw = B.transpose(1, 2).contiguous()        # (batch, nrhs, n): column-major per system
    info = torch.zeros(max(batch, 1), dtype=torch.int32, device=A.device)
    st = load().jmg_posv_batched(n, nrhs, batch, Lw.data_ptr(), max(n, 1), n * n, Xw.data_ptr(),
                                 max(n, 1), n * nrhs, dt, info.data_ptr(), _stream(A.device))
    _chk(st, "jmg_posv_batched")
    return Xw.transpose(1, 2), Lw, info[:batch]


def to_colmajor_(t: torch.Tensor, work: torch.Tensor | None = None) -> torch.Tensor:
    """Convert a contiguous row-major m x n CUDA tensor (float64 or float32) to
    column-major order IN PLACE (no second full-sized buffer) and return the
    column-major view of the same storage (same logical matrix, stride (1, m)).
    ``work``: optional device byte tensor of at least
    ``jmg_layout_workspace(m, n)`` bytes (more lets more column batches run at
    once)."""
    _need_cuda(t)
    if t.dim() != 2 or not t.is_contiguous():
        raise ValueError("to_colmajor_: a contiguous (row-major) 2-D tensor is required")
    m, n = t.shape
    dt = _dtype_code(t)
    need = int(load().jmg_layout_workspace(m, n, dt))
    if work is None:
        work = torch.empty(max(need, 256), dtype=torch.uint8, device=t.device)
    _chk(load().jmg_rowmajor_to_colmajor(m, n, t.data_ptr(), dt, work.data_ptr(), work.numel(),
                                         _stream(t.device)), "jmg_rowmajor_to_colmajor")
    return t.view(-1).view(n, m).t()


def to_rowmajor_(t: torch.Tensor, work: torch.Tensor | None = None) -> torch.Tensor:
    """The inverse of :func:`to_colmajor_`: a column-major m x n CUDA tensor
    (stride (1, m), dense) becomes row-major in place; returns the row-major
    (contiguous) view of the same storage."""
    _need_cuda(t)
    m, n = t.shape
    if t.dim() != 2 or not (t.stride(0) == 1 and (t.stride(1) == m or n == 1)):
        raise ValueError("to_rowmajor_: a dense column-major 2-D tensor is required")
    dt = _dtype_code(t)
    need = int(load().jmg_layout_workspace(n, m, dt))
    if work is None:
        work = torch.empty(max(need, 256), dtype=torch.uint8, device=t.device)
    _chk(load().jmg_colmajor_to_rowmajor(m, n, t.data_ptr(), dt, work.data_ptr(), work.numel(),
                                         _stream(t.device)), "jmg_colmajor_to_rowmajor")
    return torch.as_strided(t, (m, n), (n, 1))


def sym_grad(Bbar: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    """Abar = -(Bbar X^T + X Bbar^T) / 2 as a new n x n FP64 tensor (symmetric, so
    its row- and column-major forms coincide)."""
    _need_cuda(Bbar, X)
    pb, ldb = _colmajor(Bbar, "Bbar")
    px, ldx = _colmajor(X, "X")
    n, nrhs = X.shape
    G = torch.empty((n, n), dtype=torch.float64, device=X.device)
    _chk(load().jmg_sym_grad(n, nrhs, pb, ldb, px, ldx, G.data_ptr(), max(n, 1), _stream(X.device)),
         "jmg_sym_grad")
    return G


def logdet(L: torch.Tensor) -> torch.Tensor:
    """log det A = 2 sum log L_ii from a factor made by potrf_ (device scalar)."""
    _need_cuda(L)
    pl, lda = _colmajor(L, "L")
    out = torch.empty((), dtype=torch.float64, device=L.device)
    _chk(load().jmg_logdet(L.shape[0], pl, lda, _dtype_code(L), out.data_ptr(),
                           _stream(L.device)),
         "jmg_logdet")
    return out


def residual(A: torch.Tensor, X: torch.Tensor, B: torch.Tensor):
    """FP64 R = B - A X (lower(A) read) and per-column norms (r, x, b)."""
    _need_cuda(A, X, B)
    n, nrhs = X.shape
    pa, lda = _colmajor(A, "A")
    px, ldx = _colmajor(X, "X")
    pb, ldb = _colmajor(B, "B")
    R = torch.empty((nrhs, n), dtype=torch.float64, device=A.device).t()
    colmax = torch.zeros(3 * nrhs, dtype=torch.float64, device=A.device)
    lw = int(load().jmg_dev_residual_workspace(n, nrhs))
    work = torch.empty(max(lw, 8), dtype=torch.uint8, device=A.device)
    st = load().jmg_dev_residual(n, nrhs, pa, lda, px, ldx, pb, ldb, R.data_ptr(), n,
                                 colmax.data_ptr(), work.data_ptr(), lw, _stream(A.device))
    _chk(st, "jmg_dev_residual")
    return R, colmax.view(3, nrhs)


def residual_split(A: torch.Tensor, X: torch.Tensor, B: torch.Tensor):
    """R = B - A X with A X from the split (Ozaki) tensor-core product; also the
    per-column norms (r, x, b) and the device error word."""
    _need_cuda(A, X, B)
    n, nrhs = X.shape
    pa, lda = _colmajor(A, "A")
    px, ldx = _colmajor(X, "X")
    pb, ldb = _colmajor(B, "B")
    R = torch.empty((nrhs, n), dtype=torch.float64, device=A.device).t()
    colmax = torch.zeros(3 * nrhs, dtype=torch.float64, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    lw = int(load().jmg_dev_residual_split_workspace(n, nrhs))
    work = torch.empty(max(lw, 256), dtype=torch.uint8, device=A.device)
    st = load().jmg_dev_residual_split(n, nrhs, pa, lda, px, ldx, pb, ldb, R.data_ptr(), n,
                                       colmax.data_ptr(), err.data_ptr(), work.data_ptr(), lw,
                                       _stream(A.device))
    _chk(st, "jmg_dev_residual_split")
    return R, colmax.view(3, nrhs), err


def norm_inf(A: torch.Tensor) -> torch.Tensor:
    _need_cuda(A)
    pa, lda = _colmajor(A, "A")
    n = A.shape[0]
    out = torch.empty((), dtype=torch.float64, device=A.device)
    work = torch.empty(max(n, 1), dtype=torch.float64, device=A.device)
    st = load().jmg_dev_norm_inf(n, pa, lda, out.data_ptr(), work.data_ptr(), work.numel() * 8,
                                 _stream(A.device))
    _chk(st, "jmg_dev_norm_inf")
    return out


def syrk_tc_(C: torch.Tensor, PA: torch.Tensor, PB: torch.Tensor | None = None,
             ncols: int | None = None) -> torch.Tensor:
    """C_lower -= PA PB^T on the tensor cores (columns < ncols, default m).
    PA, PB: m x kext row-major bfloat16 or float16 (kext multiple of 64);
    C: FP32 column-major."""
    _need_cuda(C, PA)
    PB = PA if PB is None else PB
    if PA.dtype not in (torch.bfloat16, torch.float16) or PB.dtype != PA.dtype:
        raise TypeError("syrk_tc_: PA/PB must be bf16 or fp16 of one type")
    if not (PA.is_contiguous() and PB.is_contiguous()):
        raise ValueError("syrk_tc_: PA/PB must be row-major contiguous")
    m, kext = PA.shape
    pc, ldc = _colmajor(C, "C")
    err = torch.zeros(1, dtype=torch.int32, device=C.device)
    prec = PREC["bf16"] if PA.dtype == torch.bfloat16 else PREC["fp16"]
    st = load().jmg_dev_syrk_tc(m, m if ncols is None else ncols, kext, PA.data_ptr(),
                                PB.data_ptr(), kext, prec, pc, ldc, err.data_ptr(),
                                _stream(C.device))
    _chk(st, "jmg_dev_syrk_tc")
    return err


def syrk_fp8_(C: torch.Tensor, Q: torch.Tensor, e: torch.Tensor,
              ncols: int | None = None) -> torch.Tensor:
    """C_lower -= 2^-(e_i + e_j) Q_i Q_j^T (e4m3 Q: m x kext row-major bytes, e: int8
    exponent per 128-row tile; C: FP32 column-major)."""
    _need_cuda(C, Q, e)
    if Q.dtype not in (torch.uint8, getattr(torch, "float8_e4m3fn", torch.uint8)) or not Q.is_contiguous():
        raise TypeError("syrk_fp8_: Q must be contiguous e4m3 bytes")
    if e.dtype != torch.int8:
        raise TypeError("syrk_fp8_: e must be int8")
    m, kext = Q.shape
    pc, ldc = _colmajor(C, "C")
    err = torch.zeros(1, dtype=torch.int32, device=C.device)
    st = load().jmg_dev_syrk_fp8(m, m if ncols is None else ncols, kext, Q.data_ptr(), kext,
                                 e.data_ptr(), pc, ldc, err.data_ptr(), _stream(C.device))
    _chk(st, "jmg_dev_syrk_fp8")
    return err


def syrk_fp8_chunks_(C: torch.Tensor, Q: torch.Tensor, e: torch.Tensor) -> torch.Tensor:
    """C_lower -= sum_c 2^-(e[c, i] + e[c, j]) Q_i,c Q_j,c^T over 128-deep chunks c of
    K (Q: m x kext e4m3 bytes, e: (kext/128, lde) int8 exponents per chunk and
    128-row tile; C: FP32 column-major)."""
    _need_cuda(C, Q, e)
    m, kext = Q.shape
    if e.dim() != 2 or e.dtype != torch.int8 or not e.is_contiguous():
        raise TypeError("syrk_fp8_chunks_: e must be a contiguous 2-D int8 tensor")
    pc, ldc = _colmajor(C, "C")
    err = torch.zeros(1, dtype=torch.int32, device=C.device)
    st = load().jmg_dev_syrk_fp8_chunks(m, m, kext, Q.data_ptr(), kext, e.data_ptr(), e.shape[1],
                                        pc, ldc, err.data_ptr(), _stream(C.device))
    _chk(st, "jmg_dev_syrk_fp8_chunks")
    return err


def probe(kind: int, blocks: int, iters: int, device="cuda"):
    """Launch one throughput probe; returns (flops, elapsed_ms)."""
    sink = torch.zeros(max(blocks, 1), dtype=torch.float64, device=device)
    flops = ctypes.c_double(0)
    s = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    _chk(load().jmg_dev_probe(kind, blocks, iters, sink.data_ptr(), ctypes.byref(flops),
                              s.cuda_stream), "jmg_dev_probe")
    e1.record(s)
    e1.synchronize()
    return flops.value, e0.elapsed_time(e1)


def launch_count() -> int:
    return int(load().jmg_dev_launch_count())


def sv_potrs_(L: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """The mixed path's block-inverse solves on an FP32 factor: (L L^T) X = B in
    place on B (both FP32, column-major); asynchronous."""
    _need_cuda(L, B)
    if L.dtype != torch.float32 or B.dtype != torch.float32:
        raise TypeError("sv_potrs_: L and B must be float32")
    pl, lda = _colmajor(L, "L")
    pb, ldb = _colmajor(B, "B")
    n, nrhs = L.shape[0], B.shape[1]
    nbytes = int(load().jmg_dev_sv_workspace(n, nrhs))
    work = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=L.device)
    _chk(load().jmg_dev_sv_potrs(n, nrhs, pl, lda, pb, ldb, work.data_ptr(), work.numel(),
                                 _stream(L.device)), "jmg_dev_sv_potrs")
    return B


def set_wait_limit_ns(ns: int) -> int:
    """Set the time limit of every device-side wait (nanoseconds); returns the
    previous limit.  0 only queries."""
    return int(load().jmg_dev_set_wait_limit_ns(int(ns)))


def quant_fp8(L21: torch.Tensor):
    """The mixed factorisation's FP8 quantiser on its own: L21 (m x kb FP32,
    column-major) -> (Q, e): Q (m, kb) e4m3 bytes row-major (uint8), e the int8
    power-of-two exponent of each 128-row tile."""
    _need_cuda(L21)
    if L21.dtype != torch.float32:
        raise TypeError("quant_fp8: L21 must be float32")
    m, kb = L21.shape
    pl, ldw = _colmajor(L21, "L21")
    Q = torch.zeros((m, kb), dtype=torch.uint8, device=L21.device)
    e = torch.zeros(max((m + 127) // 128, 1), dtype=torch.int8, device=L21.device)
    _chk(load().jmg_dev_quant_fp8(m, kb, pl, ldw, Q.data_ptr(), kb, e.data_ptr(),
                                  _stream(L21.device)), "jmg_dev_quant_fp8")
    return Q, e[:(m + 127) // 128]
