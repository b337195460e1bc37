"""GPU parity of the FP32 storage path (potrf / potrs / posv / log det with
float32 data) against the FP64 oracle on the same (FP32-rounded) inputs.

Paper: "Software design" (potrs for float32 as well as float64 operands);
"Performance and scaling" (A = diag(1..N), b = 1, whose exact solution and
log det are known in closed form).

Tolerances follow from the arithmetic: Cholesky in precision u has backward
error bounded by a small multiple of n u, so on these well-conditioned inputs
(kappa ~ 5) the factor agrees with the exact one to c n u_32 of max|L|, and the
normwise backward error of the solve is below c n u_32 (c = 8 here).
"""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import inputs, jmg
from tests.helpers import DEV

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def dev32(M: torch.Tensor, fill=float("nan")):
    """Column-major FP32 device copy of a CPU (n x m) matrix (padding-free)."""
    n, m = M.shape
    buf = torch.full((m, n), fill, dtype=torch.float32, device=DEV)
    view = buf.t()
    view.copy_(M.to(torch.float32).to(DEV))
    return view


def host64(t: torch.Tensor) -> np.ndarray:
    return np.asfortranarray(t.detach().to(torch.float64).cpu().numpy())


def sym32(n, seed):
    """gram_shift input rounded to FP32 (the oracle sees exactly the same values)."""
    A = inputs.gram_shift(n, 1.0, seed=seed).to(torch.float32).to(torch.float64)
    return 0.5 * (A + A.t())


@pytest.mark.parametrize("nb", [64, 128])
@pytest.mark.parametrize("n", [1, 31, 128, 129, 300, 640])
def test_potrf_f32_matches_oracle(n, nb):
    A = sym32(n, inputs.seed_for("f32potrf", n))
    Lo, io = oracle.potrf(A.numpy())
    assert io == 0
    Ad = dev32(torch.tril(A) + torch.triu(torch.full_like(A, float("nan")), 1))
    info = jmg.potrf_(Ad, nb=nb)
    assert int(info.item()) == 0
    Lg = np.tril(host64(Ad))
    assert np.abs(Lg - np.tril(Lo)).max() <= 8 * max(n, 8) * U32 * np.abs(Lo).max()
    # only the lower triangle is touched (the NaN canary above it survives)
    assert np.all(np.isnan(host64(Ad)[np.triu_indices(n, 1)]))


@pytest.mark.parametrize("nrhs", [1, 16, 64, 65])
@pytest.mark.parametrize("n", [100, 257, 1000])
def test_posv_f32_backward_error(n, nrhs):
    A = sym32(n, inputs.seed_for("f32posv", n))
    B = inputs.uniform(n, nrhs, seed=nrhs).to(torch.float32).to(torch.float64)
    X, _ = jmg.posv(dev32(A), dev32(B), prec="fp64")
    assert X.dtype == torch.float32
    eta, _ = oracle.bwd_err(A.numpy(), host64(X), B.numpy())
    assert eta <= 8 * n * U32
    Xo, _ = oracle.posv(A.numpy(), B.numpy())
    assert np.abs(host64(X) - Xo).max() <= 8 * n * U32 * 5 * max(1.0, np.abs(Xo).max())


@pytest.mark.parametrize("n,nrhs", [(64, 3), (300, 17), (700, 64)])
def test_potrs_f32_with_the_oracle_factor(n, nrhs):
    A = sym32(n, inputs.seed_for("f32potrs", n))
    Lo, _ = oracle.potrf(A.numpy())
    L32 = torch.from_numpy(np.tril(Lo)).to(torch.float32).to(torch.float64)
    B = inputs.uniform(n, nrhs, seed=5).to(torch.float32).to(torch.float64)
    Xo = oracle.potrs(L32.numpy(), B.numpy())  # exact solve with the rounded factor
    Bd = dev32(B)
    jmg.potrs_(dev32(L32), Bd)
    assert np.abs(host64(Bd) - Xo).max() <= 8 * n * U32 * max(1.0, np.abs(Xo).max())


def test_logdet_f32_matches_oracle():
    n = 500
    A = sym32(n, 77)
    Ad = dev32(A)
    jmg.potrf_(Ad)
    ld = float(jmg.logdet(Ad).item())
    Lo, io = oracle.potrf(A.numpy())
    assert io == 0
    want = oracle.logdet(Lo)
    assert abs(ld - want) <= 8 * n * U32 * abs(want) + 1e-6


@pytest.mark.parametrize("N", [1000, 4096])
def test_paper_workload_diag_f32(N):
    # A = diag(1..N), b = ones: x_i = 1/i, log det = ln N!  ("Performance and scaling")
    A, b = inputs.diag_workload(N)
    X, _ = jmg.posv(dev32(A, fill=0.0), dev32(b), prec="fp64")
    x = host64(X)[:, 0]
    want = 1.0 / np.arange(1, N + 1)
    assert np.abs(x - want).max() <= 4 * U32 * want.max()
    Ad = dev32(A, fill=0.0)
    jmg.potrf_(Ad)
    assert abs(float(jmg.logdet(Ad).item()) - math.lgamma(N + 1)) <= 1e-6 * math.lgamma(N + 1)


@pytest.mark.parametrize("k", [0, 70, 200])
def test_potrf_f32_not_spd_info(k):
    n = 260
    A = sym32(n, 9)
    A[k, k] = -1.0
    _, io = oracle.potrf(A.numpy())
    info = jmg.potrf_(dev32(A), nb=64)
    assert int(info.item()) == io == k + 1


def test_mixed_modes_reject_f32():
    A = dev32(sym32(64, 1))
    B = dev32(torch.ones(64, 1, dtype=torch.float64))
    with pytest.raises(TypeError):
        jmg.posv(A, B, prec="bf16")
