"""jmg_potrs_static -- the solve with a Cholesky factor for callers that cannot
allocate device memory (fixed budgets, framework-owned pools, plain C callers
without an allocator): its scratch is a fixed array inside the library.  The
test drives it through the C ABI and compares it with jmg_potrs (which takes a
caller-provided workspace) on two calls in a row: both run the same kernels in
the same order, so the results must agree bit for bit.  It also checks that
the calls leave the device's free memory unchanged and report a clean outcome
through jmg_potrs_static_status.  It lives in a file of its own, collected
last, and needs nothing from the other tests."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import inputs, jmg

pytestmark = pytest.mark.gpu


def _dev_colmajor(M: np.ndarray) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(M.T)).to("cuda")  # rows of t = columns of M
    return t.t()  # column-major view, stride (1, rows)


def _static_call(L: torch.Tensor, B: torch.Tensor) -> int:
    lib = jmg.load()
    n, nrhs = B.shape
    return lib.jmg_potrs_static(n, nrhs, L.data_ptr(), L.stride(1), B.data_ptr(), B.stride(1),
                                jmg.JMG_F64, torch.cuda.current_stream().cuda_stream)


def _static_status() -> int:
    word = ctypes.c_int(-99)
    rc = jmg.load().jmg_potrs_static_status(ctypes.byref(word),
                                            torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    return word.value


@pytest.mark.parametrize("n,nrhs", [(1000, 5), (300, 40)])
def test_potrs_static_matches_potrs_twice(n, nrhs):
    A = inputs.gram_shift(n, 1.0, seed=inputs.seed_for("static", n)).numpy()
    L, info = oracle.potrf(A)
    assert info == 0
    L = np.tril(L)
    B = inputs.uniform(n, nrhs, seed=9).numpy()
    Ld = _dev_colmajor(L)
    # reference: the existing entry point with its caller-provided workspace
    Xref = _dev_colmajor(B)
    jmg.potrs_(Ld, Xref)
    torch.cuda.synchronize()
    ref = Xref.cpu().numpy()
    # every buffer of the calls below exists before free memory is sampled; one
    # call first so that the one-time set-up (symbol lookup) is behind us
    Xs = [_dev_colmajor(B) for _ in range(3)]
    assert _static_call(Ld, Xs[0]) == 0
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for X in Xs[1:]:  # the second call reuses the array the first one left behind
        assert _static_call(Ld, X) == 0
        torch.cuda.synchronize()
        assert _static_status() == 0
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, "the static entry point allocated device memory"
    # (the copies to the host come last: they may allocate staging buffers)
    for X in Xs:
        assert np.array_equal(X.cpu().numpy(), ref)


def test_potrs_static_rejects_oversize():
    # 65536 ints of scratch: nrhs = 512 at n = 65536 needs 1 + 32 * (2 + 2048) > 65536
    lib = jmg.load()
    rc = lib.jmg_potrs_static(65536, 512, 256, 65536, 512, 65536, jmg.JMG_F64, None)
    assert rc == 2  # JMG_ERR_WORKSPACE, nothing queued
