"""The bounded device-side waits and their abort paths.

Every spin of the library's kernels (the one-launch solves' flag waits, the
tensor-core kernels' mbarrier waits) gives up after a time limit, records the
failure and returns, so that a lost peer costs an error status, never a hung
GPU.  These tests shorten the limit to 1 ms, launch a kernel in a state where
one of its waits is never satisfied (a solve in which no CTA takes the leading
role; an update whose copy producer stays idle), and check that the kernel
returns, reports the failure, and that the next ordinary call on the same GPU
is correct.  No fault, trap or unbounded wait is involved.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import inputs, jmg
from tests.helpers import DEV, U64, host, to_dev_colmajor

pytestmark = pytest.mark.gpu

JMG_ERR_TIMEOUT = 5


@pytest.fixture
def short_waits():
    old = jmg.set_wait_limit_ns(1_000_000)  # 1 ms
    try:
        yield
    finally:
        jmg.set_wait_limit_ns(old)


def _fresh_solve_ok(n=600, nrhs=5):
    A = inputs.gram_shift(n, 1.0, seed=21)
    Lo, _ = oracle.potrf(A.numpy())
    Lo = np.tril(Lo)
    B = inputs.uniform(n, nrhs, seed=22)
    Xo = oracle.potrs(Lo, B.numpy())
    Ld, _ = to_dev_colmajor(torch.from_numpy(Lo))
    Bd, _ = to_dev_colmajor(B)
    jmg.potrs_(Ld, Bd)
    assert np.abs(host(Bd) - Xo).max() <= 64 * n * U64 * max(1.0, np.abs(Xo).max())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,nrhs", [(2048, 8), (700, 64)])
def test_solve_wait_runs_out(short_waits, dtype, n, nrhs):
    L = inputs.lower_factor(n, seed=3).to(dtype)
    B = inputs.uniform(n, nrhs, seed=4).to(dtype)
    Ld = L.to(DEV).t().contiguous().t()
    Bd = B.to(DEV).t().contiguous().t()
    code = jmg.JMG_F64 if dtype == torch.float64 else jmg.JMG_F32
    nbytes = jmg.workspace_size(jmg.OP_POTRS, n, nrhs, None, code)
    sync = torch.zeros(nbytes // 4, dtype=torch.int32, device=DEV)
    info = torch.zeros(1, dtype=torch.int32, device=DEV)
    st = jmg.load().jmg_dev_trsv_leaderless(n, nrhs, Ld.data_ptr(), n, Bd.data_ptr(), n, code,
                                            sync.data_ptr(), info.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()  # returns: every wait gave up after the limit
    assert int(sync[0].item()) == JMG_ERR_TIMEOUT
    assert int(info.item()) == -1
    # the context is intact: an ordinary solve (default limit restored below
    # only after this test; 1 ms is far above a legal wait at this size) is right
    jmg.set_wait_limit_ns(2_000_000_000)
    _fresh_solve_ok()


def test_potrs_outcome_word_is_zero_after_a_solve(short_waits):
    # jmg_potrs itself: its outcome word (work[0]) is 0 after a normal solve
    n, nrhs = 1000, 3
    L = inputs.lower_factor(n, seed=8)
    Ld = L.to(DEV).t().contiguous().t()
    Bd = inputs.uniform(n, nrhs, seed=9).to(DEV).t().contiguous().t()
    nbytes = jmg.workspace_size(jmg.OP_POTRS, n, nrhs, None)
    work = torch.full((nbytes // 4,), 77, dtype=torch.int32, device=DEV)
    jmg.set_wait_limit_ns(2_000_000_000)
    st = jmg.load().jmg_potrs(n, nrhs, Ld.data_ptr(), n, Bd.data_ptr(), n, jmg.JMG_F64,
                              work.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    assert int(work[0].item()) == 0


@pytest.mark.parametrize("m,kext", [(256, 64), (1000, 192)])
def test_tensor_core_update_wait_runs_out(short_waits, m, kext):
    g = torch.Generator().manual_seed(m)
    PA = torch.randint(-8, 9, (m, kext), generator=g).to(torch.bfloat16).to(DEV).contiguous()
    C0 = torch.randint(-100, 100, (m, m), generator=g).to(torch.float32)
    Cd = C0.to(DEV).t().contiguous().t()
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    st = jmg.load().jmg_dev_syrk_tc_idle_producer(m, m, kext, PA.data_ptr(), PA.data_ptr(), kext,
                                                  jmg.PREC["bf16"], Cd.data_ptr(), m,
                                                  err.data_ptr(),
                                                  torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    assert int(err.item()) != 0
    assert torch.equal(Cd.cpu(), C0), "an aborted update must leave C untouched"
    # the same update with its producer running is exact afterwards
    jmg.set_wait_limit_ns(2_000_000_000)
    err2 = jmg.syrk_tc_(Cd, PA)
    torch.cuda.synchronize()
    assert int(err2.item()) == 0
    want = C0.double() - PA.double().cpu() @ PA.double().cpu().t()
    lo = np.tril_indices(m)
    assert np.array_equal(Cd.double().cpu().numpy()[lo], want.numpy()[lo])
