"""Shared helpers of the GPU parity tests (input placement, oracle calls)."""
from __future__ import annotations

import numpy as np
import torch

U64 = 2.0 ** -53
DEV = "cuda"


def to_dev_colmajor(M: torch.Tensor, lda: int | None = None, fill: float | None = None):
    """Copy a CPU (n x m) matrix into a column-major device tensor with leading
    dimension lda >= n (padding rows filled with `fill`, default NaN)."""
    n, m = M.shape
    lda = lda or n
    buf = torch.full((m, lda), float("nan") if fill is None else fill, dtype=torch.float64,
                     device=DEV)
    view = buf.t()  # lda x m column-major
    view[:n, :].copy_(M.to(DEV))
    return view[:n, :], buf


def host(t: torch.Tensor) -> np.ndarray:
    return np.asfortranarray(t.detach().cpu().numpy())


def lower_sym_full(A: np.ndarray) -> np.ndarray:
    return np.tril(A) + np.tril(A, -1).T


def lower_only(A: torch.Tensor, upper_fill=float("nan")) -> torch.Tensor:
    """Copy with the strict upper triangle replaced by `upper_fill` (a canary:
    only the lower triangle may be read)."""
    B = A.clone()
    iu = torch.triu_indices(A.shape[0], A.shape[1], 1)
    B[iu[0], iu[1]] = upper_fill
    return B
