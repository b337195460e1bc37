"""Pins for the CPU oracle: checks against facts that do not come from the
oracle itself (closed forms, exact integer arithmetic, exact rationals,
independent algorithms and library routines), plus a mutation check showing
that a plausible mistake planted anywhere in oracle.c fails at least one pin.

Paper: "Software design" (potrs = Cholesky potrf + potrs, optional log det);
"Performance and scaling" (benchmark matrix A = diag(1..N), b = ones).
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import inputs

U64 = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_3x3():
    rows = []
    with open(os.path.join(GOLDEN, "cholesky_3x3.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows[:3]), np.array(rows[3:6])


def _spd(n, seed, shift=1.0):
    return inputs.gram_shift(n, shift, seed).numpy()


def _full(A):
    """symmetric matrix from its lower triangle"""
    L = np.tril(A)
    return L + np.tril(A, -1).T


# ----------------------------------------------------------------------------- pins


def pin_textbook(o):
    A, Lg = _golden_3x3()
    L, info = o.potrf(A)
    assert info == 0
    assert np.array_equal(np.tril(L), Lg)
    # upper triangle never referenced: passed through unchanged
    assert np.array_equal(np.triu(L, 1), np.triu(A, 1))


def pin_integer_factor(o):
    for n, seed in [(1, 0), (2, 5), (7, 1), (24, 2), (40, 3)]:
        Lt, A = inputs.integer_factor(n, seed)
        Lt, A = Lt.numpy(), A.numpy()
        L, info = o.potrf(A)
        assert info == 0
        assert np.array_equal(np.tril(L), Lt), n


def pin_diag_closed_form(o):
    # A = diag(1..N), b = ones: L = diag(sqrt(i)), x_i = 1/i, log det = ln N!
    N = 50
    A, b = inputs.diag_workload(N)
    A, b = A.numpy(), b.numpy()
    L, info = o.potrf(A)
    assert info == 0
    assert np.count_nonzero(np.tril(L, -1)) == 0
    d = np.diag(L)
    i = np.arange(1, N + 1, dtype=np.float64)
    assert np.all(np.abs(d * d - i) <= 4 * U64 * i)
    x, info = o.posv(A, b)
    assert info == 0
    assert np.all(np.abs(x[:, 0] - 1.0 / i) <= 4 * U64 / i)
    ld = o.logdet(L)
    assert abs(ld - math.lgamma(N + 1)) <= 1e-13 * math.lgamma(N + 1)


def pin_ge_agrees(o):
    # GE with partial pivoting vs the Cholesky solve vs LAPACK (numpy), n <= 12.
    rng = np.random.default_rng(7)
    for n in (1, 2, 5, 12):
        # widely varying diagonal so that partial pivoting actually swaps rows
        D = np.diag(np.logspace(0, 4, n)[::-1] if n > 1 else [1.0])
        A = D @ _spd(n, 11 + n) @ D
        B = rng.standard_normal((n, 3))
        Xc, ic = o.posv(A, B)
        Xg, ig = o.ge_solve(A, B)
        Xn = np.linalg.solve(_full(A), B)
        assert ic == 0 and ig == 0
        kappa = np.linalg.cond(_full(A))
        tol = 50 * kappa * U64
        scale = np.abs(Xn).max()
        assert np.abs(Xc - Xn).max() <= tol * scale, (n, "chol")
        assert np.abs(Xg - Xn).max() <= tol * scale, (n, "ge")


def pin_ge_pivots(o):
    # A 2x2 SPD matrix whose elimination without the row swap would use the
    # tiny pivot: [[eps, 1], [1, 2]] is not SPD, so use a symmetric one where
    # |a_10| > |a_00|: [[1, 3], [3, 10]] (det 1 > 0); x = A^{-1} b exactly.
    A = np.array([[1.0, 3.0], [3.0, 10.0]])
    b = np.array([[1.0], [2.0]])
    x, info = o.ge_solve(A, b)
    assert info == 0
    # exact inverse [[10, -3], [-3, 1]]
    assert np.allclose(x[:, 0], [10 * 1 - 3 * 2, -3 * 1 + 1 * 2], rtol=0, atol=4 * U64 * 10)


def pin_known_solution(o):
    # b = A x_true; forward error within kappa * u, backward error ~ u.
    n, kappa = 96, 1e6
    A = inputs.q_lambda(n, kappa, seed=3).numpy()
    Xt = inputs.uniform(n, 4, seed=4).numpy()
    B = A @ Xt
    X, info = o.posv(A, B)
    assert info == 0
    fwd = np.abs(X - Xt).max() / np.abs(Xt).max()
    assert fwd <= 10 * kappa * n * U64
    eta, _ = o.bwd_err(A, X, B)
    assert eta <= 20 * U64


def pin_scipy_cholesky(o):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    for n in (3, 33, 70):
        A = _spd(n, 20 + n)
        L, info = o.potrf(A)
        Ls = scipy_linalg.cholesky(_full(A), lower=True)
        assert info == 0
        assert np.abs(np.tril(L) - Ls).max() <= 8 * n * U64 * np.abs(Ls).max()


def pin_potrs_residual(o):
    # (L L^T) X = B checked with plain matrix products
    rng = np.random.default_rng(3)
    n = 40
    L = np.tril(rng.uniform(-0.5, 0.5, (n, n)), -1) + np.diag(rng.uniform(1.0, 2.0, n))
    B = rng.standard_normal((n, 5))
    X = o.potrs(L, B)
    R = B - L @ (L.T @ X)
    assert np.abs(R).max() <= 200 * n * U64 * np.abs(B).max()


def pin_dot2_exact(o):
    # Sums with heavy cancellation: plain FP64 loses every digit, Dot2 must be
    # as accurate as a twice-the-precision computation rounded once.
    rng = np.random.default_rng(5)
    n = 9
    for trial in range(6):
        e = rng.integers(-30, 30, size=(n, n))
        A = np.ldexp(rng.uniform(0.5, 1.0, (n, n)), e)
        A = np.tril(A) + np.tril(A, -1).T
        X = np.ldexp(rng.uniform(-1, 1, (n, 2)), rng.integers(-30, 30, size=(n, 2)))
        # choose B so that the residual is small compared to the terms
        B = np.array(_full(A) @ X)
        B += np.ldexp(rng.uniform(-1, 1, B.shape), -40)
        R = o.resid_dot2(A, X, B)
        Af = _full(A)
        for c in range(X.shape[1]):
            for i in range(n):
                exact = Fraction(B[i, c]) - sum(Fraction(Af[i, j]) * Fraction(X[j, c])
                                                 for j in range(n))
                big = sum(abs(Fraction(Af[i, j]) * Fraction(X[j, c])) for j in range(n))
                err = abs(Fraction(R[i, c]) - exact)
                assert err <= Fraction(U64) * abs(exact) + Fraction(2.0 ** -100) * big, (trial, i)


def pin_bwd_err_formula(o):
    rng = np.random.default_rng(9)
    n = 6
    A = np.tril(rng.integers(-9, 10, (n, n)).astype(float))
    A = A + np.diag(np.full(n, 40.0))
    X = rng.integers(-5, 6, (n, 3)).astype(float)
    E = rng.integers(-3, 4, (n, 3)).astype(float)
    E[:, 0] = 0.0  # column 0 solved exactly: the maximum must come from another column
    E[0, 2] = 5.0
    B = _full(A) @ X + E  # exact integers
    eta, per = o.bwd_err(A, X, B)
    assert per[0] == 0.0 and eta > 0.0
    Af = _full(A)
    anorm = np.abs(Af).sum(axis=1).max()
    assert o.norm_inf(A) == anorm
    R = B - Af @ X  # exact (small integers)
    for c in range(3):
        want = np.abs(R[:, c]).max() / (anorm * np.abs(X[:, c]).max() + np.abs(B[:, c]).max())
        assert abs(per[c] - want) <= 4 * U64 * want
    assert eta == per.max()


def pin_not_spd(o):
    A = _spd(10, 1)
    for k in (0, 3, 9):
        Ak = A.copy()
        Ak[k, k] = -1.0
        _, info = o.potrf(Ak)
        assert info == k + 1
        Ak[k, k] = np.nan
        _, info = o.potrf(Ak)
        assert info == k + 1
    _, info = o.potrf(np.zeros((3, 3)))
    assert info == 1
    # singular PSD: second pivot is exactly zero
    _, info = o.potrf(np.array([[1.0, 1.0], [1.0, 1.0]]))
    assert info == 2


def pin_logdet_library(o):
    for n in (1, 8, 30):
        A = _spd(n, 40 + n, shift=0.5)
        L, info = o.potrf(A)
        sign, ref = np.linalg.slogdet(_full(A))
        assert info == 0 and sign > 0
        assert abs(o.logdet(L) - ref) <= 1e-12 * max(1.0, abs(ref))


def _loss(o, A, B):
    X, info = o.posv(A, B)
    assert info == 0
    return 0.5 * float(np.sum(X * X))


def pin_grad_fd(o):
    # loss = 0.5 ||X||_F^2, X = A^{-1} B, Xbar = X.  The symmetric,
    # half-weighted perturbation A + h (e_i e_j^T + e_j e_i^T)/2 has directional
    # derivative exactly Abar_ij = -(Bbar X^T + X Bbar^T)_ij / 2.
    n, nrhs, h = 6, 2, 1e-5
    A = _spd(n, 2)
    B = np.random.default_rng(1).standard_normal((n, nrhs))
    X0, _ = o.posv(A, B)
    X, Bbar, Abar, info = o.grad(A, B, X0)
    assert info == 0
    assert np.abs(X - X0).max() <= 0.0
    assert np.array_equal(Abar, Abar.T)
    for i in range(n):
        for j in range(i + 1):
            # only lower(A) is read, so +h on the stored entry (i, j), i > j,
            # moves both a_ij and a_ji: twice the half-weighted direction.
            E = np.zeros((n, n))
            E[i, j] = 1.0
            fd = (_loss(o, A + h * E, B) - _loss(o, A - h * E, B)) / (2 * h)
            want = Abar[i, j] * (1.0 if i == j else 2.0)
            assert abs(fd - want) <= 1e-6 * max(1.0, abs(want)), (i, j)
    for i in range(n):
        for c in range(nrhs):
            Bp, Bm = B.copy(), B.copy()
            Bp[i, c] += h
            Bm[i, c] -= h
            fd = (_loss(o, A, Bp) - _loss(o, A, Bm)) / (2 * h)
            assert abs(fd - Bbar[i, c]) <= 1e-6 * max(1.0, abs(Bbar[i, c]))


def pin_grad_library(o):
    # torch autograd through LAPACK's solve on sym(S): gradient w.r.t. S equals
    # the symmetric Abar.
    n, nrhs = 5, 3
    A = _spd(n, 8)
    B = np.random.default_rng(2).standard_normal((n, nrhs))
    S = torch.tensor(_full(A), requires_grad=True)
    Bt = torch.tensor(B, requires_grad=True)
    Xt = torch.linalg.solve(0.5 * (S + S.T), Bt)
    (0.5 * (Xt * Xt).sum()).backward()
    X, Bbar, Abar, info = o.grad(A, B, Xt.detach().numpy())
    assert info == 0
    assert np.abs(Abar - S.grad.numpy()).max() <= 1e-12 * max(1.0, np.abs(Abar).max())
    assert np.abs(Bbar - Bt.grad.numpy()).max() <= 1e-12 * max(1.0, np.abs(Bbar).max())


def pin_bwd_err_rows_bit_identical(o):
    # the cache-friendly sweep computes every residual entry and row sum with
    # the same operations in the same order as the plain definition, so it must
    # agree bit for bit (ragged row blocks, one and several right-hand sides, a
    # NaN, a zero right-hand side)
    for n, nrhs, seed in [(1, 1, 0), (31, 1, 1), (33, 3, 2), (100, 7, 3), (257, 2, 4)]:
        A = inputs.q_lambda(n, 1e6, seed) if n > 1 else np.array([[2.0]])
        A = np.asarray(A)
        X = np.random.default_rng(seed).uniform(-1, 1, (n, nrhs))
        B = np.asfortranarray(_full(A) @ X + 1e-9 * np.random.default_rng(seed + 9).standard_normal((n, nrhs)))
        if nrhs > 2:
            B[:, 1] = 0.0
            X[:, 1] = 0.0
        w1, e1 = o.bwd_err(A, X, B)
        w2, e2 = o.bwd_err_rows(A, X, B)
        assert w1 == w2 and np.array_equal(e1, e2), (n, nrhs)
    A = _spd(40, 5)
    X = np.ones((40, 2))
    X[7, 1] = np.nan
    B = _full(A) @ np.ones((40, 2))
    w1, e1 = o.bwd_err(A, X, B)
    w2, e2 = o.bwd_err_rows(A, X, B)
    assert np.isnan(w1) and np.isnan(w2) and e1[0] == e2[0] and np.isnan(e2[1])


def pin_layout_conversion(o):
    # worked example by hand: the 2 x 3 matrix [[1, 2, 3], [4, 5, 6]] held
    # row-major is [1 2 3 4 5 6]; column-major it is [1 4 2 5 3 6]
    assert np.array_equal(o.rowmajor_to_colmajor(np.array([1., 2, 3, 4, 5, 6]), 2, 3),
                          np.array([1., 4, 2, 5, 3, 6]))
    # and NumPy's own column-major flattening of the same matrix
    for m, n in [(1, 7), (7, 1), (5, 5), (6, 10), (13, 4)]:
        M = np.random.default_rng(m * 31 + n).standard_normal((m, n))
        assert np.array_equal(o.rowmajor_to_colmajor(M.reshape(-1), m, n), M.reshape(-1, order="F"))


PINS = [pin_textbook, pin_integer_factor, pin_diag_closed_form, pin_ge_agrees, pin_ge_pivots,
        pin_known_solution, pin_scipy_cholesky, pin_potrs_residual, pin_dot2_exact,
        pin_bwd_err_formula, pin_not_spd, pin_logdet_library, pin_grad_fd, pin_grad_library,
        pin_bwd_err_rows_bit_identical, pin_layout_conversion]


@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_oracle_pin(pin):
    pin(oracle.default())


# ------------------------------------------------------------------ planted mistakes

MUTANTS = {
    "no_sqrt": ("double ljj = sqrt(d);", "double ljj = d;"),
    "update_sign": ("AT(A, i, k, lda) -= AT(A, i, j, lda) * lkj;",
                    "AT(A, i, k, lda) += AT(A, i, j, lda) * lkj;"),
    "update_skips_diag": ("for (int i = k; i < n; ++i) AT(A, i, k, lda) -=",
                          "for (int i = k + 1; i < n; ++i) AT(A, i, k, lda) -="),
    "no_scale": ("AT(A, i, j, lda) = AT(A, i, j, lda) / ljj;", "AT(A, i, j, lda) = AT(A, i, j, lda);"),
    "back_transposed": ("s -= AT(L, i, j, lda) * b[i];", "s -= AT(L, j, i, lda) * b[i];"),
    "forward_sign": ("b[i] -= AT(L, i, j, lda) * yj;", "b[i] += AT(L, i, j, lda) * yj;"),
    "back_no_divide": ("b[j] = s / AT(L, j, j, lda);", "b[j] = s;"),
    "dot2_drop_prod_err": ("comp += es + ep;", "comp += es;"),
    "dot2_drop_sum_err": ("comp += es + ep;", "comp += ep;"),
    "twosum_wrong": ("*e = (a - (x - z)) + (b - z);", "*e = (a - (x - z));"),
    "norm_no_abs": ("s += fabs(sym_at(A, lda, i, j));", "s += sym_at(A, lda, i, j);"),
    "sym_at_upper": ("return i >= j ? AT(A, i, j, lda) : AT(A, j, i, lda);",
                     "return AT(A, i, j, lda);"),
    "bwd_no_b": ("double den = anorm * xn + bn;", "double den = anorm * xn;"),
    "nan_not_caught": ("if (!(d > 0.0)) return j + 1;", "if (d <= 0.0) return j + 1;"),
    "info_off_by_one": ("if (!(d > 0.0)) return j + 1;", "if (!(d > 0.0)) return j;"),
    "logdet_no_two": ("return 2.0 * s;", "return s;"),
    "grad_half_missing": ("AT(Abar, i, j, ldab) = -0.5 * s;", "AT(Abar, i, j, ldab) = -1.0 * s;"),
    "grad_one_term": ("s += Bbar[(size_t)c * n + i] * X[(size_t)c * n + j] +\n"
                      "             X[(size_t)c * n + i] * Bbar[(size_t)c * n + j];",
                      "s += 2.0 * Bbar[(size_t)c * n + i] * X[(size_t)c * n + j];"),
    "grad_sign": ("AT(Abar, i, j, ldab) = -0.5 * s;", "AT(Abar, i, j, ldab) = 0.5 * s;"),
    "ge_no_rhs_swap": ("AT(B, k, c, ldb) = AT(B, p, c, ldb);\n        AT(B, p, c, ldb) = t;",
                       "(void)t;"),
    "ge_back_index": ("s -= M[(size_t)j * n + i] * AT(B, j, c, ldb);",
                      "s -= M[(size_t)i * n + j] * AT(B, j, c, ldb);"),
    "forward_no_divide": ("double yj = b[j] / AT(L, j, j, lda);", "double yj = b[j];"),
    "update_skips_next_col": ("for (int k = j + 1; k < n; ++k) {\n      double lkj",
                              "for (int k = j + 2; k < n; ++k) {\n      double lkj"),
    "twoprod_sign": ("*e = fma(a, b, -x);", "*e = fma(a, b, x);"),
    "resid_sign": ("two_prod(-sym_at(A, lda, i, j), AT(X, j, c, ldx), &p, &ep);",
                   "two_prod(sym_at(A, lda, i, j), AT(X, j, c, ldx), &p, &ep);"),
    "resid_lower_row_only": ("      for (int j = 0; j < n; ++j) {\n        double p, ep, es;",
                             "      for (int j = 0; j <= i; ++j) {\n        double p, ep, es;"),
    "norm_lower_row_only": ("for (int j = 0; j < n; ++j) s += fabs(sym_at(A, lda, i, j));",
                            "for (int j = 0; j <= i; ++j) s += fabs(sym_at(A, lda, i, j));"),
    "norm_sums_rows": ("if (s > best || isnan(s)) best = s;", "best += s;"),
    "bwd_first_column_only": ("if (e > worst || isnan(e)) worst = e;", "if (c == 0) worst = e;"),
    "bwd_x_from_b": ("xn = nan_max(xn, fabs(AT(X, i, c, ldx)));",
                     "xn = nan_max(xn, fabs(AT(B, i, c, ldb)));"),
    "grad_uses_b": ("Bbar[(size_t)c * n + i] = AT(Xbar, i, c, ldxb);",
                    "Bbar[(size_t)c * n + i] = AT(B, i, c, ldb);"),
    "logdet_no_log": ("s += log(AT(L, i, i, lda));", "s += AT(L, i, i, lda);"),
    "rows_drop_prod_err": ("comp[(size_t)ii * nr + c] += es + ep;",
                           "comp[(size_t)ii * nr + c] += es;"),
    "rows_norm_no_abs": ("asum[ii] += fabs(a);", "asum[ii] += a;"),
    "rows_lower_only": ("const double a = sym_at(A, lda, i0 + ii, j);",
                        "const double a = j <= i0 + ii ? sym_at(A, lda, i0 + ii, j) : 0.0;"),
    "layout_transposed": ("out[i + j * m] = in[i * n + j];", "out[i * n + j] = in[i + j * m];"),
    # planted mistakes stay inside the buffers: the mutant runs in this process
    "layout_no_move": ("out[i + j * m] = in[i * n + j];", "out[i * n + j] = in[i * n + j];"),
    "rows_skip_tail": ("const int ib = n - i0 < ORACLE_ROWS ? n - i0 : ORACLE_ROWS;",
                       "const int ib = n - i0 < ORACLE_ROWS ? n - i0 - 1 : ORACLE_ROWS;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) >= 1, name
    o = oracle.variant(src.replace(old, new, 1), str(tmp_path))
    failed = []
    for pin in PINS:
        try:
            pin(o)
        except Exception:  # AssertionError or a numerical blow-up
            failed.append(pin.__name__)
    assert failed, "mutant %s passes every pin" % name
