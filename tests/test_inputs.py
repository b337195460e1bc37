"""CPU checks of the seeded input recipe: each generator produces the matrix
class it states (spectrum, symmetry, exactness, layout) and is reproducible
from its seed.  These are the workloads every parity test and the bench draw
from."""
from __future__ import annotations

import math

import numpy as np
import torch

from paper_2601_14466_gb300 import inputs


def test_q_lambda_has_the_stated_spectrum():
    for n, kappa in ((64, 1e6), (200, 1e2), (150, 1e8)):
        A = inputs.q_lambda(n, kappa, seed=inputs.seed_for("inputs", n))
        assert torch.equal(A, A.t())  # exactly symmetric
        ev = np.linalg.eigvalsh(A.numpy())
        want = kappa ** (np.arange(n) / (n - 1))
        # eigenvalues of Q diag(lambda) Q^T are lambda up to rounding of the products
        assert np.abs(ev - want).max() <= 1e3 * n * 2.0 ** -53 * kappa
        assert abs(ev[-1] / ev[0] / kappa - 1.0) <= 1e-6 * max(1.0, kappa * 1e-8)
    assert inputs.q_lambda(1, 1e6).item() == 1.0


def test_gram_shift_is_spd_with_the_marchenko_pastur_range():
    n = 300
    A = inputs.gram_shift(n, 1.0, seed=5)
    assert torch.equal(A, A.t())
    ev = np.linalg.eigvalsh(A.numpy())
    # eig(M M^T / n) lies in [0, ~4] for square M: kappa <= ~5 with shift 1
    assert ev[0] >= 1.0 - 1e-12 and ev[-1] <= 5.5
    A2 = inputs.gram_shift(n, 1e-2, seed=5)
    ev2 = np.linalg.eigvalsh(A2.numpy())
    assert ev2[0] >= 1e-2 - 1e-12 and ev2[-1] / ev2[0] > 50  # a few hundred
    # the FP32-product variant stays exactly symmetric and positive definite
    A3 = inputs.gram_shift(n, 1.0, seed=5, fp32_product=True)
    assert torch.equal(A3, A3.t()) and np.linalg.eigvalsh(A3.numpy())[0] > 0.99


def test_diag_workload_and_its_closed_forms():
    N = 50
    A, b = inputs.diag_workload(N)
    assert torch.equal(A, torch.diag(torch.arange(1, N + 1, dtype=torch.float64)))
    assert b.shape == (N, 1) and b.stride(0) == 1 and torch.all(b == 1.0)
    # x_i = 1 / i and log det A = ln N!
    assert abs(float(torch.log(torch.diagonal(A)).sum()) - math.lgamma(N + 1)) < 1e-10


def test_integer_factor_is_exact():
    L, A = inputs.integer_factor(40, seed=3)
    Li = L.to(torch.int64)
    assert torch.equal(Li.to(torch.float64), L) and torch.equal(torch.tril(Li), Li)
    d = torch.diagonal(Li)
    assert torch.all((d > 0) & ((d & (d - 1)) == 0))  # powers of two
    assert torch.equal((Li @ Li.t()).to(torch.float64), A)


def test_layout_ranges_and_products():
    X = inputs.uniform(37, 5, seed=2)
    assert X.shape == (37, 5) and X.stride() == (1, 37)
    assert float(X.min()) >= -1.0 and float(X.max()) <= 1.0
    Y = inputs.normal(37, 5, seed=2)
    assert Y.stride() == (1, 37)
    A = inputs.gram_shift(37, 1.0, seed=1)
    B = inputs.rhs_from(A, X)
    assert B.stride() == (1, 37) and torch.equal(B, A @ X)
    assert inputs.nominal_flops(3, 2) == 9.0 + 36.0


def test_seeds_reproduce_and_separate():
    assert torch.equal(inputs.q_lambda(32, 1e3, seed=7), inputs.q_lambda(32, 1e3, seed=7))
    assert not torch.equal(inputs.uniform(8, 2, seed=1), inputs.uniform(8, 2, seed=2))
    assert inputs.seed_for("posv", 100, 1e6) == inputs.seed_for("posv", 100, 1e6)
    assert inputs.seed_for("posv", 100) != inputs.seed_for("posv", 101)
    assert 0 <= inputs.seed_for("x") < 2 ** 31
