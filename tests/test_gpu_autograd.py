"""Differentiation of the SPD solve: the hand-written adjoint against
gradcheck (tiny n), the oracle's gradient and central finite differences with
the FP64 forward (paper: "Summary" -- potrs composes with the framework's
transformations; gradient Abar = -(Bbar X^T + X Bbar^T)/2)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import autograd, inputs, jmg
from tests.helpers import DEV

pytestmark = pytest.mark.gpu


def _sym(S):
    return 0.5 * (S + S.mT)


@pytest.mark.parametrize("n,nrhs", [(1, 1), (5, 2), (9, 3)])
def test_gradcheck_fp64(n, nrhs):
    g = torch.Generator().manual_seed(n)
    M = torch.randn(n, n, generator=g, dtype=torch.float64)
    S0 = (M @ M.T / n + torch.eye(n, dtype=torch.float64)).to(DEV).requires_grad_(True)
    B0 = torch.randn(n, nrhs, generator=g, dtype=torch.float64).to(DEV).requires_grad_(True)
    # sym() makes every perturbation of S a symmetric one, as the solver reads one triangle
    f = lambda S, B: autograd.solve(_sym(S), B, "fp64")  # noqa: E731
    assert torch.autograd.gradcheck(f, (S0, B0), eps=1e-6, atol=1e-7, rtol=1e-6)


@pytest.mark.parametrize("prec,words", [("fp64", 1), ("bf16", 2), ("fp16", 1)])
def test_grad_matches_oracle(prec, words):
    n, nrhs = 600, 16
    A = inputs.gram_shift(n, 1.0, seed=21)
    B = inputs.normal(n, nrhs, seed=22)
    Ad = A.to(DEV).requires_grad_(True)
    Bd = B.to(DEV).requires_grad_(True)
    X = autograd.solve(Ad, Bd, prec, words)
    loss = 0.5 * (X * X).sum()
    loss.backward()
    Xo, Bbo, Abo, info = oracle.grad(A.numpy(), B.numpy(), oracle.posv(A.numpy(), B.numpy())[0])
    assert info == 0
    # kappa ~ 5: both gradients agree to ~1e-12 of their scale (mixed: within the refinement tol)
    tol = 1e-11 if prec == "fp64" else 1e-10
    ga, gb = Ad.grad.cpu().numpy(), Bd.grad.cpu().numpy()
    assert np.abs(ga - Abo).max() <= tol * np.abs(Abo).max()
    assert np.abs(gb - Bbo).max() <= tol * np.abs(Bbo).max()
    assert np.array_equal(ga, ga.T)


def _loss_fp64(Ad, Bd):
    X, _ = jmg.posv(Ad, Bd, prec="fp64")
    return 0.5 * float((X * X).sum().item())


@pytest.mark.parametrize("n,nrhs,count", [(300, 4, 12), (8192, 16, 64)])
def test_grad_central_differences(n, nrhs, count):
    # config of the differentiation workload at full size: n=8192, nrhs=16,
    # A = M M^T/n + I, B ~ N(0,1), loss 0.5||X||^2, h = 1e-6, 64 random entries
    A = inputs.gram_shift(n, 1.0, seed=31, device=DEV)
    B = inputs.normal(n, nrhs, seed=32, device=DEV)
    Ad = A.clone().requires_grad_(True)
    X = autograd.solve(Ad, B, "bf16", 2)  # mixed forward; FD below uses the FP64 forward
    (0.5 * (X * X).sum()).backward()
    G = Ad.grad
    rng = np.random.default_rng(33)
    h = 1e-6
    for _ in range(count):
        i, j = sorted(rng.integers(0, n, size=2))[::-1]
        E = torch.zeros_like(A)
        # symmetric perturbation of the pair (i, j): +h on both entries (one for i == j)
        E[i, j] = h
        E[j, i] = h
        fd = (_loss_fp64((A + E).mT, B) - _loss_fp64((A - E).mT, B)) / (2 * h)
        want = float(G[i, j] + G[j, i]) if i != j else float(G[i, i])
        assert abs(fd - want) <= 1e-4 * max(1.0, abs(want)), (i, j, fd, want)
