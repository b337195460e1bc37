"""The mixed path's block-inverse triangular solves (forward L Y = B, back
L^T X = Y with the FP32 factor) against the oracle's substitution.

The solves run through jmg_dev_sv_potrs on a directly drawn, well-conditioned
FP32 factor: the inverses of the 128 x 128 diagonal blocks are formed in FP64,
the chain multiplies by them and by the coupling blocks Li L_{b,b-e}, and the
helper CTAs stream the blocks of L by TMA from the factor mirrored into its
upper triangle.  The oracle solves the same FP32-rounded system in FP64, so
the difference is FP32 arithmetic only.  Sizes span one block, ragged tails,
several right-hand-side groups (16 per leader, 64 per launch) and a launch in
which helpers take several tickets each.  Paper: "Software design" (potrs)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import inputs, jmg
from tests.helpers import DEV, host

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _run(n, nrhs, seed):
    L = inputs.lower_factor(n, seed=seed).to(torch.float32)
    B = inputs.uniform(n, nrhs, seed=seed + 1).to(torch.float32)
    Xo = oracle.potrs(L.double().numpy(), B.double().numpy())
    Ld = L.to(DEV).t().contiguous().t()
    Bd = B.to(DEV).t().contiguous().t()
    jmg.sv_potrs_(Ld, Bd)
    torch.cuda.synchronize()
    return host(Bd).astype(np.float64), Xo


@pytest.mark.parametrize("n", [1, 5, 127, 128, 129, 300, 384, 385, 1000, 2100])
@pytest.mark.parametrize("nrhs", [1, 3, 16, 17, 33, 64, 65, 130])
def test_sv_potrs_matches_oracle(n, nrhs):
    Xg, Xo = _run(n, nrhs, seed=inputs.seed_for("sv", n, nrhs))
    # FP32 arithmetic (block inverses formed in FP64, rounded to FP32): the
    # bound is 2^11 ulps of max|X|; a block product lost or applied twice
    # moves entries at O(1e-2)
    assert np.abs(Xg - Xo).max() <= 2048 * U32 * max(1.0, np.abs(Xo).max())


@pytest.mark.parametrize("nrhs", [1, 32, 64])
def test_sv_potrs_full_size(nrhs):
    Xg, Xo = _run(16384, nrhs, seed=77 + nrhs)
    assert np.abs(Xg - Xo).max() <= 2048 * U32 * max(1.0, np.abs(Xo).max())


@pytest.mark.parametrize("n,nrhs", [(2100, 33), (2100, 64), (4000, 20)])
def test_sv_potrs_is_deterministic(n, nrhs):
    # every CTA adds its products in a fixed order, so repeated solves of the
    # same system agree bit for bit; a race between the CTAs' roles (a block
    # read before it is published, a buffer reused too early) shows up here
    L = inputs.lower_factor(n, seed=11).to(torch.float32).to(DEV).t().contiguous().t()
    B = inputs.uniform(n, nrhs, seed=12).to(torch.float32).to(DEV)
    first = None
    for _ in range(6):
        Bd = jmg.colmajor_copy(B)  # a fresh copy: the solve works in place
        jmg.sv_potrs_(L, Bd)
        torch.cuda.synchronize()
        got = Bd.cpu()
        if first is None:
            first = got
        else:
            assert torch.equal(got, first)
