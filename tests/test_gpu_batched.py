"""GPU parity of the batched small-system path (jmg_posv_batched) against the
CPU oracle, system by system.  Paper: "Summary" -- potrs as a primitive that
composes with the framework's transformations, including vectorisation over a
batch of systems."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import inputs, jmg
from tests.helpers import DEV, U64

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _systems(batch, n, nrhs, seed):
    As = [inputs.gram_shift(n, 1.0, seed=seed + b) for b in range(batch)]
    Bs = [inputs.uniform(n, nrhs, seed=seed + 1000 + b) for b in range(batch)]
    return torch.stack(As), torch.stack(Bs)


@pytest.mark.parametrize("n,nrhs,batch", [(1, 1, 3), (5, 2, 17), (64, 1, 40), (100, 70, 9),
                                          (128, 16, 12)])
def test_posv_batched_matches_oracle(n, nrhs, batch):
    A, B = _systems(batch, n, nrhs, seed=inputs.seed_for("batched", n))
    X, _, info = jmg.posv_batched(A.to(DEV), B.to(DEV))
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0] * batch
    Xh = X.cpu().numpy()
    for b in range(batch):
        Xo, io = oracle.posv(A[b].numpy(), B[b].numpy())
        assert io == 0
        assert np.abs(Xh[b] - Xo).max() <= 64 * max(n, 8) * U64 * max(1.0, np.abs(Xo).max())


def test_posv_batched_info_per_system():
    n, nrhs, batch = 50, 3, 6
    A, B = _systems(batch, n, nrhs, seed=7)
    A[2, 10, 10] = -1.0  # system 2 is not positive definite at its 11th minor
    Ad, Bd = A.to(DEV), B.to(DEV)
    X, _, info = jmg.posv_batched(Ad, Bd)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0, 11, 0, 0, 0]
    assert torch.equal(X[2].cpu(), B[2])  # the failed system keeps its right-hand side
    for b in (0, 5):
        Xo, _ = oracle.posv(A[b].numpy(), B[b].numpy())
        assert np.abs(X[b].cpu().numpy() - Xo).max() <= 1e-12 * max(1.0, np.abs(Xo).max())


def test_posv_batched_f32():
    n, nrhs, batch = 96, 4, 10
    A, B = _systems(batch, n, nrhs, seed=11)
    A32, B32 = A.to(torch.float32), B.to(torch.float32)
    X, _, info = jmg.posv_batched(A32.to(DEV), B32.to(DEV))
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0] * batch
    for b in range(batch):
        A64, B64 = A32[b].double(), B32[b].double()
        eta, _ = oracle.bwd_err(A64.numpy(), np.asfortranarray(X[b].double().cpu().numpy()),
                                B64.numpy())
        assert eta <= 8 * n * U32


def test_posv_batched_factors():
    n, batch = 40, 4
    A, B = _systems(batch, n, 1, seed=3)
    _, L, info = jmg.posv_batched(A.to(DEV), B.to(DEV))
    torch.cuda.synchronize()
    for b in range(batch):
        Lg = np.tril(L[b].cpu().numpy().T)
        Lo, _ = oracle.potrf(A[b].numpy())
        assert np.abs(Lg - np.tril(Lo)).max() <= 64 * n * U64 * np.abs(Lo).max()
