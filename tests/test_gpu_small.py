"""The one-kernel mixed posv for small systems (prec "fp32": FP32 tile
Cholesky, FP64 residual and the refinement's stopping rule on the device)
against the oracle.  Paper: "Software design" (potrs as one call) and the
refinement of Section 3.

Every solution is certified by the oracle's Dot2 backward error and compared
with the oracle's FP64 solve; the kernel's own backward error must agree with
the oracle's; the result is bitwise reproducible (tile products are added in a
fixed order); A is left untouched (NaN canary in its upper triangle)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import inputs, jmg
from tests.helpers import U64, host, lower_only, to_dev_colmajor

pytestmark = pytest.mark.gpu

JMG_ERR_NOT_SPD, JMG_ERR_TIMEOUT, JMG_ERR_UNSUPPORTED = 3, 5, 6


def _solve_check(A, B, kappa, tol=1e-13, **kw):
    Ad, _ = to_dev_colmajor(lower_only(A))
    A_before = Ad.clone()
    Bd, _ = to_dev_colmajor(B)
    X, si = jmg.posv(Ad, Bd, prec="fp32", tol=tol, **kw)
    assert si.status == 0 and si.info == 0, si
    Xg = host(X)
    eta, _ = oracle.bwd_err(A.numpy(), Xg, B.numpy())
    assert eta <= tol, eta
    # the device's backward error is the same quantity (plain FP64 products)
    assert si.bwd_err <= tol and abs(si.bwd_err - eta) <= 0.05 * tol + 8 * A.shape[0] * U64, \
        (si.bwd_err, eta)
    Xo, io = oracle.posv(A.numpy(), B.numpy())
    assert io == 0
    bound = 40 * kappa * max(tol, U64) * np.abs(Xo).max()
    assert np.abs(Xg - Xo).max() <= bound
    assert torch.equal(torch.nan_to_num(Ad, nan=7.0), torch.nan_to_num(A_before, nan=7.0))
    return X, si


@pytest.mark.parametrize("n,nrhs", [(1, 1), (17, 2), (64, 1), (65, 3), (130, 1), (700, 4),
                                    (1024, 1), (1024, 16), (1500, 9), (2048, 8), (2000, 64)])
def test_small_posv_gram(n, nrhs):
    A = inputs.gram_shift(n, 1.0, seed=inputs.seed_for("small", n))
    B = inputs.rhs_from(A, inputs.uniform(n, nrhs, seed=7))
    _, si = _solve_check(A, B, kappa=10.0)
    assert si.factor_tries == 1 and si.iters <= 4


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
def test_small_posv_kappa(kappa):
    n = 900
    A = inputs.q_lambda(n, kappa, seed=inputs.seed_for("small-q", n))
    B = inputs.rhs_from(A, inputs.uniform(n, 3, seed=8))
    _solve_check(A, B, kappa=kappa)


def test_small_posv_deterministic_and_one_launch():
    n, nrhs = 1111, 5
    A = inputs.gram_shift(n, 1.0, seed=31)
    B = inputs.rhs_from(A, inputs.uniform(n, nrhs, seed=32))
    Ad, _ = to_dev_colmajor(lower_only(A))
    Bd, _ = to_dev_colmajor(B)
    work = jmg.workspace(jmg.OP_POSV, n, nrhs, jmg.default_options(prec="fp32"), "cuda")
    c0 = jmg.launch_count()
    X1, s1 = jmg.posv(Ad, Bd, prec="fp32", work=work)
    assert jmg.launch_count() - c0 == 1  # the whole solve is one kernel
    X2, s2 = jmg.posv(Ad, Bd, prec="fp32", work=work)
    assert torch.equal(X1, X2) and s1.iters == s2.iters and s1.bwd_err == s2.bwd_err


def test_small_posv_not_spd():
    n = 300
    A = inputs.gram_shift(n, 1.0, seed=2)
    A[100, 100] = -50.0
    Ad, _ = to_dev_colmajor(A)
    Bd, _ = to_dev_colmajor(inputs.uniform(n, 1, seed=1))
    _, si = jmg.posv(Ad, Bd, prec="fp32", shift_retry=False, check=False)
    assert si.status == JMG_ERR_NOT_SPD and si.info == 101


def test_small_posv_shift_retry():
    # kappa 1e9 breaks the FP32 factor; the kernel shifts the diagonal by
    # 4 u_32 max|a_ii| (then 16x) and factors again, on the device
    n = 512
    A = inputs.q_lambda(n, 1e9, seed=inputs.seed_for("small-shift", n))
    B = inputs.rhs_from(A, inputs.uniform(n, 2, seed=9))
    Ad, _ = to_dev_colmajor(A)
    Bd, _ = to_dev_colmajor(B)
    X, si = jmg.posv(Ad, Bd, prec="fp32", check=False, maxit=100)
    assert si.factor_tries >= 2 and si.shift > 0.0
    assert si.status in (0, 4)
    if si.status == 0:
        eta, _ = oracle.bwd_err(A.numpy(), host(X), B.numpy())
        assert eta <= 1e-13


def test_small_posv_limits():
    for n, nrhs in [(2049, 1), (100, 65)]:
        A = inputs.gram_shift(n, 1.0, seed=3)
        Ad, _ = to_dev_colmajor(A)
        Bd, _ = to_dev_colmajor(inputs.uniform(n, nrhs, seed=4))
        with pytest.raises(jmg.JmgError) as e:
            jmg.posv(Ad, Bd, prec="fp32")
        assert e.value.status == JMG_ERR_UNSUPPORTED


def test_small_posv_wait_runs_out():
    # a 1 ns limit: the first grid barrier or tile wait gives up, the kernel
    # records the timeout and every CTA leaves; the next call is correct
    n = 640
    A = inputs.gram_shift(n, 1.0, seed=41)
    B = inputs.rhs_from(A, inputs.uniform(n, 2, seed=42))
    Ad, _ = to_dev_colmajor(A)
    Bd, _ = to_dev_colmajor(B)
    old = jmg.set_wait_limit_ns(1)
    try:
        _, si = jmg.posv(Ad, Bd, prec="fp32", check=False)
    finally:
        jmg.set_wait_limit_ns(old)
    assert si.status == JMG_ERR_TIMEOUT
    _solve_check(A, B, kappa=10.0)


def test_small_posv_nan_rhs_stops():
    # a NaN in B makes its residual NaN: the device-side rule stops at the first
    # check (no refinement steps) and reports NOT_CONVERGED; the other columns
    # are unaffected by the bad one only through the shared stopping decision
    n = 300
    A = inputs.gram_shift(n, 1.0, seed=51)
    B = inputs.rhs_from(A, inputs.uniform(n, 2, seed=52))
    B[7, 1] = float("nan")
    Ad, _ = to_dev_colmajor(A)
    Bd, _ = to_dev_colmajor(B)
    X, si = jmg.posv(Ad, Bd, prec="fp32", check=False)
    assert si.status == 4  # JMG_ERR_NOT_CONVERGED
    assert si.iters == 0 and np.isnan(si.bwd_err)
    assert np.isnan(host(X)[:, 1]).any()
