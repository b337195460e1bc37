"""Seeded synthetic inputs for the SPD solve path.

This module holds no arithmetic of the method (no factorisation, no solve): it
only draws matrices and right-hand sides.  Both the CUDA path's tests and the
CPU oracle consume what it makes, so it is kept apart from each of them.

Workloads (column-major FP64, ``lda = n``; symmetric matrices are returned with
both triangles filled, so a row-major tensor is also its own column-major
form):

* ``gram_shift``  A = M M^T / n + s I with M i.i.d. N(0,1)  (s = 1 gives
  kappa ~ 5; s = 1e-2 gives kappa of a few hundred: eig(M M^T / n) lies in
  [~0, 4] for square M, Marchenko-Pastur with ratio 1).
* ``q_lambda``   A = Q diag(lambda) Q^T, Q from the Householder QR of an
  i.i.d. N(0,1) matrix with the signs fixed so that diag(R) > 0, lambda
  log-spaced in [1, kappa] (kappa_2(A) = kappa up to rounding).
* ``diag_workload``  A = diag(1, ..., N), b = (1, ..., 1)^T, the benchmark
  matrix of the paper ("Performance and scaling").
* ``integer_factor``  a random integer lower-triangular L_true with power-of-two
  diagonal and A = L_true L_true^T formed exactly: every step of a Cholesky
  factorisation of A is exact in FP64, so the factor must come back bit for bit.

The dense generators run on whatever ``device`` is given (QR and products go
through torch's own linear algebra, which is input preparation only).
"""
from __future__ import annotations

import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def col_major(n: int, m: int, *, dtype=torch.float64, device="cpu") -> torch.Tensor:
    """An uninitialised n x m column-major tensor (stride (1, n))."""
    return torch.empty((m, n), dtype=dtype, device=device).t()


def gram_shift(n: int, shift: float, seed: int = 0, device="cpu", fp32_product: bool = False
               ) -> torch.Tensor:
    """A = M M^T / n + shift I.  fp32_product draws M and forms the product in
    FP32 (then widens to FP64): for n in the tens of thousands the FP64
    product alone would take minutes on a GPU with slow FP64.  The matrix is
    still exactly symmetric and, for shift >> n u_32, positive definite."""
    g = _gen(seed, device)
    if fp32_product:
        M = torch.randn((n, n), generator=g, dtype=torch.float32, device=device)
        A32 = M @ M.t()
        del M
        A = A32.to(torch.float64)
        del A32
    else:
        M = torch.randn((n, n), generator=g, dtype=torch.float64, device=device)
        A = M @ M.t()
        del M
    A.div_(n)
    A = 0.5 * (A + A.t())
    A.diagonal().add_(shift)
    return A.contiguous()


def q_factor(n: int, seed: int = 0, device="cpu") -> torch.Tensor:
    """Q of the Householder QR of an i.i.d. N(0,1) n x n matrix, with the signs
    fixed so that diag(R) > 0 (a Haar-distributed orthogonal matrix)."""
    g = _gen(seed, device)
    G = torch.randn((n, n), generator=g, dtype=torch.float64, device=device)
    Q, R = torch.linalg.qr(G)
    del G
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1.0
    Q.mul_(s.unsqueeze(0))
    return Q


def from_q(Q: torch.Tensor, kappa: float) -> torch.Tensor:
    """A = Q diag(lambda) Q^T with lambda log-spaced in [1, kappa], symmetrised.
    Several condition numbers can share one (expensive) Q."""
    n = Q.shape[0]
    lam = log_spaced(n, kappa, device=Q.device)
    QL = Q * lam.unsqueeze(0)
    # the product block by block, lower blocks only, mirrored (A is symmetric;
    # this skips ~40% of the FP64 multiply work of a full product)
    A = torch.empty((n, n), dtype=Q.dtype, device=Q.device)
    nb = 8
    cuts = [n * k // nb for k in range(nb + 1)]
    for bi in range(nb):
        r0, r1 = cuts[bi], cuts[bi + 1]
        for bj in range(bi + 1):
            c0, c1 = cuts[bj], cuts[bj + 1]
            blk = QL[r0:r1] @ Q[c0:c1].t()
            A[r0:r1, c0:c1] = blk
            if bj < bi:
                A[c0:c1, r0:r1] = blk.t()
    del QL
    A = 0.5 * (A + A.t())
    return A.contiguous()


def q_lambda(n: int, kappa: float, seed: int = 0, device="cpu") -> torch.Tensor:
    return from_q(q_factor(n, seed, device), kappa)


def log_spaced(n: int, kappa: float, device="cpu") -> torch.Tensor:
    """lambda_i = kappa^{i/(n-1)}, i = 0..n-1 (ascending, lambda_0 = 1)."""
    if n == 1:
        return torch.ones(1, dtype=torch.float64, device=device)
    t = torch.arange(n, dtype=torch.float64, device=device) / (n - 1)
    return torch.pow(torch.tensor(float(kappa), dtype=torch.float64, device=device), t)


def diag_workload(n: int, device="cpu"):
    """A = diag(1..n), b = ones(n, 1)."""
    A = torch.diag(torch.arange(1, n + 1, dtype=torch.float64, device=device))
    b = col_major(n, 1, device=device)
    b.fill_(1.0)
    return A, b


def uniform(n: int, m: int, seed: int = 0, device="cpu", lo=-1.0, hi=1.0) -> torch.Tensor:
    """n x m column-major, i.i.d. U[lo, hi]."""
    g = _gen(seed, device)
    X = torch.rand((m, n), generator=g, dtype=torch.float64, device=device)
    X.mul_(hi - lo).add_(lo)
    return X.t()


def normal(n: int, m: int, seed: int = 0, device="cpu") -> torch.Tensor:
    """n x m column-major, i.i.d. N(0, 1)."""
    g = _gen(seed, device)
    return torch.randn((m, n), generator=g, dtype=torch.float64, device=device).t()


def rhs_from(A: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    """B = A X (FP64 matrix product of the generator; column-major result)."""
    B = col_major(X.shape[0], X.shape[1], device=X.device)
    B.copy_(A @ X)
    return B


def integer_factor(n: int, seed: int = 0, max_abs: int = 8, max_exp: int = 3):
    """(L_true, A): L_true lower triangular with integer entries in
    [-max_abs, max_abs] below the diagonal and diagonal 2^e, e in [0, max_exp];
    A = L_true L_true^T computed exactly (all partial sums are integers far
    below 2^53)."""
    g = _gen(seed, "cpu")
    L = torch.randint(-max_abs, max_abs + 1, (n, n), generator=g, dtype=torch.int64)
    L = torch.tril(L, -1)
    e = torch.randint(0, max_exp + 1, (n,), generator=g, dtype=torch.int64)
    L = L + torch.diag(torch.pow(2, e))
    A = L @ L.t()  # exact in int64
    assert int(A.abs().max()) < 2 ** 52
    return L.to(torch.float64), A.to(torch.float64)


def lower_factor(n: int, seed: int = 0, device="cpu") -> torch.Tensor:
    """A well-conditioned lower-triangular factor for solve-only tests (no
    factorisation needed): strictly lower entries i.i.d. N(0, 1/n), diagonal
    2 + U[0, 1].  Row i's off-diagonal part has 2-norm about sqrt(i/n) <= 1,
    so forward and back substitution keep |y| of the order of |b| and every
    block product changes the result at O(1).  Column-major, upper triangle 0."""
    g = _gen(seed, device)
    L = torch.randn((n, n), generator=g, dtype=torch.float64, device=device)
    L.mul_(n ** -0.5)
    L = torch.tril(L, -1)
    d = torch.rand(n, generator=g, dtype=torch.float64, device=device)
    L.diagonal().copy_(2.0 + d)
    return L.t().contiguous().t()


def nominal_flops(n: int, nrhs: int) -> float:
    """n^3/3 + 2 n^2 nrhs: the usual count for one Cholesky solve."""
    return n ** 3 / 3.0 + 2.0 * n * n * nrhs


def seed_for(*parts) -> int:
    """Stable seed from a tuple of labels (no Python hash randomisation)."""
    h = 1469598103934665603
    for p in parts:
        for ch in str(p).encode():
            h = ((h ^ ch) * 1099511628211) % (1 << 63)
    return int(h % (1 << 31))


