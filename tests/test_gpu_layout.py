"""The in-place row-major -> column-major conversion (paper: "Local
memory-layout conversion") against the oracle's plain definition.

The conversion moves elements without arithmetic, so the result must equal the
oracle's out-of-place rewrite bit for bit: shapes with gcd(m, n) > 1 (the
column rotation runs) and = 1 (it does not), vectors, rows longer than shared
memory holds (the scratch-row path), a scratch buffer that holds only one
column batch at a time, FP32 and FP64, and the inverse move back."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import jmg
from tests.helpers import DEV

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n", [(1, 9), (9, 1), (2, 3), (64, 64), (96, 64), (100, 37),
                                 (1000, 24), (24, 1000), (3000, 64), (257, 1031), (512, 768)])
def test_rowmajor_to_colmajor_matches_oracle(m, n, dtype):
    g = torch.Generator().manual_seed(m * 1009 + n)
    M = torch.randn((m, n), generator=g, dtype=torch.float64).to(dtype)
    t = M.to(DEV).contiguous()
    C = jmg.to_colmajor_(t)
    torch.cuda.synchronize()
    got = t.view(-1).cpu().double().numpy()  # the buffer itself, now column-major
    want = oracle.rowmajor_to_colmajor(M.double().numpy().reshape(-1), m, n)
    assert np.array_equal(got, want)
    assert C.stride() == (1, m) and torch.equal(C.cpu(), M)
    # and back
    R = jmg.to_rowmajor_(C)
    torch.cuda.synchronize()
    assert R.is_contiguous() and torch.equal(R.cpu(), M)


def test_long_rows_and_small_scratch():
    # rows of 30000 doubles (240 KB) take the scratch-row path; the scratch holds
    # exactly one column batch, so every batch reuses it in turn
    m, n = 48, 30000
    M = torch.randn((m, n), generator=torch.Generator().manual_seed(3), dtype=torch.float64)
    t = M.to(DEV).contiguous()
    need = int(jmg.load().jmg_layout_workspace(m, n, jmg.JMG_F64))
    work = torch.empty(need, dtype=torch.uint8, device=DEV)
    C = jmg.to_colmajor_(t, work=work)
    torch.cuda.synchronize()
    want = oracle.rowmajor_to_colmajor(M.numpy().reshape(-1), m, n)
    assert np.array_equal(t.view(-1).cpu().numpy(), want)
    assert torch.equal(C.cpu(), M)


def test_full_size_right_hand_sides():
    # the right-hand sides of the n = 65536, nrhs = 32 workload, row-major as a
    # framework holds them, converted in place for the solver
    m, n = 65536, 32
    M = torch.randn((m, n), generator=torch.Generator().manual_seed(5), dtype=torch.float64)
    t = M.to(DEV).contiguous()
    C = jmg.to_colmajor_(t)
    torch.cuda.synchronize()
    assert torch.equal(C.cpu(), M)
    assert np.array_equal(t.view(-1).cpu().numpy(), M.numpy().reshape(-1, order="F"))
