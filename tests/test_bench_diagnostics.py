"""CPU check of bench.py's componentwise (Oettli-Prager) backward-error
diagnostic: the formula max_ij |r_ij| / (|A| |x_j| + |b_j|)_i on a small exact
example, the zero-denominator cases, and that a failing residual call yields
None instead of an exception.  The library's residual is replaced by an exact
CPU one (no GPU here)."""
from __future__ import annotations

import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _ExactResidual:
    def residual_split(self, Acm, X, B):
        R = B - Acm.t() @ X  # A symmetric: the lower triangle stands for the whole
        return R, None, torch.zeros(1, dtype=torch.int32)


class _Failing:
    def residual_split(self, Acm, X, B):
        raise RuntimeError("no device")


def test_componentwise_formula():
    A = torch.tensor([[4.0, -1.0, 0.0], [-1.0, 3.0, 2.0], [0.0, 2.0, 5.0]], dtype=torch.float64)
    X = torch.tensor([[1.0, 0.5], [2.0, -1.0], [-1.0, 0.25]], dtype=torch.float64)
    B = A @ X
    B[1, 0] += 0.125   # row 1 of column 0 off by 1/8
    B[2, 1] -= 0.5     # row 2 of column 1 off by 1/2
    got = bench._cw_bwd_err(_ExactResidual(), torch, A, A.t(), X, B)
    D = A.abs() @ X.abs() + B.abs()
    want = max(0.125 / float(D[1, 0]), 0.5 / float(D[2, 1]))
    assert abs(got - want) <= 1e-15 * want
    # exact solution: zero; a zero row with a non-zero residual: infinite
    assert bench._cw_bwd_err(_ExactResidual(), torch, A, A.t(), X, A @ X) == 0.0
    Z = torch.zeros(3, 3, dtype=torch.float64)
    Xz = torch.zeros(3, 1, dtype=torch.float64)
    Bz = torch.tensor([[0.0], [1.0], [0.0]], dtype=torch.float64)
    assert bench._cw_bwd_err(_ExactResidual(), torch, Z, Z, Xz, Bz) == 1.0  # |r| / |b| = 1
    Bz0 = torch.zeros(3, 1, dtype=torch.float64)
    assert bench._cw_bwd_err(_ExactResidual(), torch, Z, Z, Xz, Bz0) == 0.0


def test_componentwise_failure_is_none():
    A = torch.eye(4, dtype=torch.float64)
    X = torch.ones(4, 1, dtype=torch.float64)
    assert bench._cw_bwd_err(_Failing(), torch, A, A, X, X) is None

    class _Shape:  # above n = 16384 the diagnostic is not taken
        shape = (16385, 16385)

    assert bench._cw_bwd_err(_ExactResidual(), torch, _Shape(), None, None, None) is None
