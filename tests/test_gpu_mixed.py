"""Mixed-precision posv (tensor-core factor + FP64 refinement) against the
oracle: backward error certified by the oracle's Dot2 residual, solution
compared with the oracle's FP64 solve within a kappa-scaled bound, and A left
untouched.  Paper: "Software design" (potrs semantics)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import inputs, jmg
from tests.helpers import U64, host, lower_only, to_dev_colmajor

pytestmark = pytest.mark.gpu


def _check(A, B, X, kappa, tol=1e-13):
    Xg = host(X)
    eta, _ = oracle.bwd_err(A.numpy(), Xg, B.numpy())
    assert eta <= tol, eta
    Xo, io = oracle.posv(A.numpy(), B.numpy())
    assert io == 0
    # both solutions have backward error <= tol: they differ by <= ~2 kappa tol
    bound = 4 * kappa * max(tol, U64) * np.abs(Xo).max() * 10
    assert np.abs(Xg - Xo).max() <= bound
    return eta


@pytest.mark.parametrize("prec,words", [("bf16", 1), ("bf16", 2), ("bf16", 3), ("fp16", 1),
                                        ("fp16", 2)])
@pytest.mark.parametrize("n,nrhs", [(64, 3), (130, 1), (257, 2), (700, 4), (1100, 16)])
def test_posv_mixed_gram(prec, words, n, nrhs):
    A = inputs.gram_shift(n, 1.0, seed=inputs.seed_for("mixed", n))
    Xt = inputs.uniform(n, nrhs, seed=5)
    B = inputs.rhs_from(A, Xt)
    Ad, _ = to_dev_colmajor(lower_only(A))
    A_before = Ad.clone()
    Bd, _ = to_dev_colmajor(B)
    X, si = jmg.posv(Ad, Bd, prec=prec, words=words)
    assert si.status == 0 and si.info == 0
    assert si.bwd_err <= 1e-13
    _check(A, B, X, kappa=10.0)
    # A is preserved bit for bit (NaN canary in the upper triangle included)
    assert torch.equal(torch.nan_to_num(Ad, nan=7.0), torch.nan_to_num(A_before, nan=7.0))


@pytest.mark.parametrize("n", [100, 640, 1001])
def test_posv_mixed_nb64(n):
    # 64-wide panels: the diagonal factor, the panel solve and the split update
    # at half width (and the overlap of the next diagonal block with the rest)
    A = inputs.gram_shift(n, 1.0, seed=inputs.seed_for("nb64", n))
    Xt = inputs.uniform(n, 5, seed=6)
    B = inputs.rhs_from(A, Xt)
    Ad, _ = to_dev_colmajor(lower_only(A))
    Bd, _ = to_dev_colmajor(B)
    X, si = jmg.posv(Ad, Bd, prec="bf16", words=2, nb=64)
    assert si.status == 0 and si.info == 0
    assert si.bwd_err <= 1e-13
    _check(A, B, X, kappa=10.0)


@pytest.mark.parametrize("kappa,prec,words", [(1e2, "bf16", 1), (1e4, "bf16", 2),
                                              (1e4, "fp16", 1), (1e6, "bf16", 3)])
def test_posv_mixed_q_lambda(kappa, prec, words):
    n, nrhs = 1000, 4
    A = inputs.q_lambda(n, kappa, seed=inputs.seed_for("qlam", kappa))
    Xt = inputs.uniform(n, nrhs, seed=6)
    B = inputs.rhs_from(A, Xt)
    Ad, _ = to_dev_colmajor(lower_only(A))
    Bd, _ = to_dev_colmajor(B)
    X, si = jmg.posv(Ad, Bd, prec=prec, words=words, maxit=60)
    assert si.status == 0, si
    _check(A, B, X, kappa)


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_posv_leaves_inputs_alone(prec):
    # posv returns a new X: neither B nor (without overwrite_a) A may change,
    # also when they are already column-major
    n, nrhs = 300, 5
    A = inputs.gram_shift(n, 1.0, seed=12)
    B = inputs.uniform(n, nrhs, seed=13)
    Ad, _ = to_dev_colmajor(A)
    Bd, _ = to_dev_colmajor(B)
    A0, B0 = Ad.clone(), Bd.clone()
    X, _ = jmg.posv(Ad, Bd, prec=prec)
    X2, _ = jmg.posv(Ad, Bd, prec=prec)
    assert torch.equal(Ad, A0) and torch.equal(Bd, B0)
    assert X.data_ptr() != Bd.data_ptr()
    assert torch.allclose(X, X2, rtol=1e-12, atol=0)


@pytest.mark.parametrize("refine", ["pcg", "auto"])
@pytest.mark.parametrize("kappa,prec,words", [(1e6, "bf16", 3), (1e8, "bf16", 3), (1e8, "fp16", 2)])
def test_posv_mixed_high_kappa(kappa, prec, words, refine):
    # kappa * u_factor >= 1: stationary refinement alone stalls; PCG preconditioned
    # by the (possibly diagonally shifted) factor must still reach 1e-13
    n, nrhs = 1000, 3
    A = inputs.q_lambda(n, kappa, seed=inputs.seed_for("hk", kappa))
    Xt = inputs.uniform(n, nrhs, seed=7)
    B = inputs.rhs_from(A, Xt)
    Ad, _ = to_dev_colmajor(lower_only(A))
    Bd, _ = to_dev_colmajor(B)
    X, si = jmg.posv(Ad, Bd, prec=prec, words=words, refine=refine, maxit=200)
    assert si.status == 0, si
    _check(A, B, X, kappa)


@pytest.mark.parametrize("n,nrhs,shift", [(700, 4, 1e-2), (2000, 8, 1e-2), (1500, 2, 1.0)])
def test_posv_fp8_tile_scaled(n, nrhs, shift):
    # e4m3 trailing updates with one power-of-two scale per 128 x 128 panel
    # tile, FP64 refinement (PCG and the diagonal shift as needed) to 1e-13
    A = inputs.gram_shift(n, shift, seed=inputs.seed_for("fp8", n))
    Xt = inputs.uniform(n, nrhs, seed=8)
    B = inputs.rhs_from(A, Xt)
    Ad, _ = to_dev_colmajor(lower_only(A))
    Bd, _ = to_dev_colmajor(B)
    X, si = jmg.posv(Ad, Bd, prec="fp8", maxit=300)
    assert si.status == 0, si
    _check(A, B, X, kappa=1e3)


def test_posv_reuse_factor():
    # a refine-only call with the factor left in the workspace by a first call
    n, nrhs = 700, 3
    A = inputs.gram_shift(n, 1e-2, seed=41)
    B1 = inputs.uniform(n, nrhs, seed=42)
    B2 = inputs.normal(n, nrhs + 2, seed=43)
    Ad, _ = to_dev_colmajor(A)
    work = jmg.workspace(jmg.OP_POSV, n, nrhs + 2, jmg.default_options(prec="bf16", words=2),
                         "cuda")
    X1, s1 = jmg.posv(Ad, to_dev_colmajor(B1)[0], prec="bf16", words=2, work=work)
    X2, s2 = jmg.posv(Ad, to_dev_colmajor(B2)[0], prec="bf16", words=2, work=work,
                      reuse_factor=True)
    assert s1.factor_tries == 1 and s2.factor_tries == 0
    _check(A, B1, X1, kappa=500.0)
    _check(A, B2, X2, kappa=500.0)


def test_posv_mixed_not_spd():
    n = 300
    A = inputs.gram_shift(n, 1.0, seed=2)
    A[100, 100] = -50.0
    Ad, _ = to_dev_colmajor(A)
    Bd, _ = to_dev_colmajor(inputs.uniform(n, 1, seed=1))
    X, si = jmg.posv(Ad, Bd, prec="bf16", shift_retry=False, check=False)
    assert si.status == 3  # JMG_ERR_NOT_SPD
    assert si.info == 101
