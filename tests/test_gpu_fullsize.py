"""Parity at the benchmark's sizes.

The one-launch solves hand blocks to helper CTAs by tickets; once a launch has
fewer CTAs than blocks (n = 16384 and up, as in the benchmark), helpers take a
second and third ticket.  These tests reach that path and compare the GPU
solves element by element with the oracle's substitution on a directly drawn,
well-conditioned factor (no oracle factorisation needed), in FP64 and FP32
storage.  A mixed-precision posv at n = 12288 (FP16 x 2 words, kappa = 1e6) is
certified by the oracle's Dot2 backward error and compared with the oracle's
FP64 solve.  Paper: "Software design" (potrs)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import inputs, jmg
from tests.helpers import DEV, U64, host

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _dev(M: torch.Tensor, dtype) -> torch.Tensor:
    return M.to(dtype).to(DEV).t().contiguous().t()


@pytest.fixture(scope="module")
def factor16k():
    n = 16384
    L = inputs.lower_factor(n, seed=inputs.seed_for("fullsize", n))
    return n, L


@pytest.mark.parametrize("nrhs", [1, 64])
def test_potrs_fp64_full_size(factor16k, nrhs):
    n, L = factor16k
    B = inputs.uniform(n, nrhs, seed=nrhs)
    Xo = oracle.potrs(L.numpy(), B.numpy())
    Bd = _dev(B, torch.float64)
    jmg.potrs_(_dev(L, torch.float64), Bd)
    Xg = host(Bd)
    # FP64 substitution on a well-conditioned factor: ~1e2 ulps of |X|; a block
    # product lost or applied twice moves entries at O(1e-2)
    assert np.abs(Xg - Xo).max() <= 2048 * U64 * max(1.0, np.abs(Xo).max())


@pytest.mark.parametrize("nrhs", [1, 64])
def test_potrs_fp32_full_size(factor16k, nrhs):
    n, L = factor16k
    B = inputs.uniform(n, nrhs, seed=100 + nrhs)
    # the oracle solves the FP32-rounded system exactly enough (FP64)
    L32 = L.to(torch.float32)
    B32 = B.to(torch.float32)
    Xo = oracle.potrs(L32.double().numpy(), B32.double().numpy())
    Bd = _dev(B32, torch.float32)
    jmg.potrs_(_dev(L32, torch.float32), Bd)
    Xg = host(Bd).astype(np.float64)
    # FP32 arithmetic: a column-by-column FP32 substitution of the same system
    # is off by ~1e2 ulps of |X| at this n; bound 2^11 ulps
    assert np.abs(Xg - Xo).max() <= 2048 * U32 * max(1.0, np.abs(Xo).max())


def test_posv_mixed_fp16x2_n12288_kappa1e6():
    n, nrhs, kappa = 12288, 4, 1e6
    A = inputs.q_lambda(n, kappa, seed=inputs.seed_for("fullsize-mixed", n), device=DEV)
    Xt = inputs.uniform(n, nrhs, seed=7, device=DEV)
    B = inputs.rhs_from(A, Xt)
    X, si = jmg.posv(A.t(), B, prec="fp16", words=2)
    assert si.status == 0, si
    Ah = np.asfortranarray(A.cpu().numpy())
    Bh = host(B)
    Xg = host(X)
    eta, _ = oracle.bwd_err(Ah, Xg, Bh)
    assert eta <= 1e-13, eta
    Xo, io = oracle.posv(Ah, Bh)
    assert io == 0
    # both have backward error <= 1e-13 on a kappa = 1e6 system
    assert np.abs(Xg - Xo).max() <= 40 * kappa * 1e-13 * np.abs(Xo).max()
