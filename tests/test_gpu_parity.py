"""GPU parity of the FP64 path and the building blocks against the CPU oracle.

Element by element at sizes the oracle finishes in seconds, spanning several
64/128 blocks and ragged tails.  Paper: "Software design" (potrs = potrf +
potrs, optional log det); "Performance and scaling" (A = diag(1..N), b = 1).
"""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import inputs, jmg
from tests.helpers import DEV, U64, host, lower_only, lower_sym_full, to_dev_colmajor

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 31, 64, 65, 127, 128, 129, 300, 515]


@pytest.mark.parametrize("nb", [64, 128])
@pytest.mark.parametrize("n", SIZES)
def test_potrf_matches_oracle(n, nb):
    A = inputs.gram_shift(n, 1.0, seed=inputs.seed_for("potrf", n))
    Ad, _ = to_dev_colmajor(lower_only(A))
    info = jmg.potrf_(Ad, nb=nb)
    assert int(info.item()) == 0
    Lg = np.tril(host(Ad))
    Lo, io = oracle.potrf(A.numpy())
    assert io == 0
    Lo = np.tril(Lo)
    # well conditioned (kappa ~ 5): elementwise agreement to a few ulps of ||L||
    assert np.abs(Lg - Lo).max() <= 64 * max(n, 8) * U64 * np.abs(Lo).max()
    # the strict upper triangle was a NaN canary and must be untouched
    up = host(Ad)[np.triu_indices(n, 1)]
    assert np.all(np.isnan(up))


@pytest.mark.parametrize("n", [7, 64, 129, 200])
def test_potrf_exact_integer_factor(n):
    # every operation is exact in FP64 (integers, power-of-two pivots): bit-exact
    Lt, A = inputs.integer_factor(n, seed=n)
    Ad, _ = to_dev_colmajor(A)
    info = jmg.potrf_(Ad, nb=64)
    assert int(info.item()) == 0
    assert np.array_equal(np.tril(host(Ad)), Lt.numpy())


def test_potrf_padding_and_lda():
    n, lda = 257, 300
    A = inputs.gram_shift(n, 1.0, seed=3)
    Ad, buf = to_dev_colmajor(lower_only(A), lda=lda)
    info = jmg.potrf_(Ad, nb=128)
    assert int(info.item()) == 0
    pad = buf.t()[n:, :].cpu().numpy()
    assert np.all(np.isnan(pad)), "padding rows n..lda-1 were written"
    Lo, _ = oracle.potrf(A.numpy())
    assert np.abs(np.tril(host(Ad)) - np.tril(Lo)).max() <= 1e-13 * np.abs(Lo).max()


@pytest.mark.parametrize("k", [0, 5, 63, 64, 130, 299])
def test_potrf_not_spd_info(k):
    n = 300
    A = inputs.gram_shift(n, 1.0, seed=9)
    A[k, k] = -1.0
    _, io = oracle.potrf(A.numpy())
    Ad, _ = to_dev_colmajor(A)
    info = jmg.potrf_(Ad, nb=64)
    assert int(info.item()) == io == k + 1
    A[k, k] = float("nan")
    Ad, _ = to_dev_colmajor(A)
    info = jmg.potrf_(Ad, nb=128)
    assert int(info.item()) == k + 1


@pytest.mark.parametrize("nrhs", [1, 3, 16, 33, 64])
@pytest.mark.parametrize("n", [1, 100, 128, 257, 640, 2100])
def test_potrs_matches_oracle(n, nrhs):
    A = inputs.gram_shift(n, 1.0, seed=inputs.seed_for("potrs", n))
    Lo, _ = oracle.potrf(A.numpy())
    Lo = np.tril(Lo)
    B = inputs.uniform(n, nrhs, seed=nrhs)
    Xo = oracle.potrs(Lo, B.numpy())
    Ld, _ = to_dev_colmajor(torch.from_numpy(Lo))
    Bd, _ = to_dev_colmajor(B)
    jmg.potrs_(Ld, Bd)
    Xg = host(Bd)
    assert np.abs(Xg - Xo).max() <= 64 * n * U64 * max(1.0, np.abs(Xo).max())


@pytest.mark.parametrize("kappa", [1e2, 1e6])
@pytest.mark.parametrize("n,nrhs", [(200, 2), (1024, 1), (777, 16)])
def test_posv_fp64_backward_error(n, nrhs, kappa):
    A = inputs.q_lambda(n, kappa, seed=inputs.seed_for("posv", n, kappa))
    Xt = inputs.uniform(n, nrhs, seed=1)
    B = inputs.rhs_from(A, Xt)
    Ad, _ = to_dev_colmajor(lower_only(A))
    Bd, _ = to_dev_colmajor(B)
    X, si = jmg.posv(Ad, Bd, prec="fp64")
    Xg = host(X)
    eta, _ = oracle.bwd_err(A.numpy(), Xg, B.numpy())
    assert eta <= 1e-13, eta
    Xo, _ = oracle.posv(A.numpy(), B.numpy())
    assert np.abs(Xg - Xo).max() <= 100 * kappa * n * U64 * np.abs(Xo).max()
    fwd = np.abs(Xg - Xt.numpy()).max() / np.abs(Xt.numpy()).max()
    assert fwd <= 10 * kappa * max(eta, U64) * n


def test_paper_workload_diag():
    # A = diag(1..N), b = ones: x_i = 1/i, log det = ln N!  ("Performance and scaling")
    N = 1000
    A, b = inputs.diag_workload(N)
    Ad, _ = to_dev_colmajor(A)
    bd, _ = to_dev_colmajor(b)
    info = jmg.potrf_(Ad)
    assert int(info.item()) == 0
    ld = float(jmg.logdet(Ad).item())
    jmg.potrs_(Ad, bd)
    i = np.arange(1, N + 1, dtype=np.float64)
    assert np.all(np.abs(host(bd)[:, 0] - 1.0 / i) <= 4 * U64 / i)
    assert abs(ld - math.lgamma(N + 1)) <= 1e-12 * math.lgamma(N + 1)


def test_logdet_matches_oracle():
    n = 300
    A = inputs.gram_shift(n, 0.5, seed=4)
    Lo, _ = oracle.potrf(A.numpy())
    Ld, _ = to_dev_colmajor(torch.from_numpy(np.tril(Lo)))
    assert abs(float(jmg.logdet(Ld).item()) - oracle.logdet(Lo)) <= 1e-12 * abs(oracle.logdet(Lo))


@pytest.mark.parametrize("n,nrhs", [(1, 1), (70, 3), (300, 17), (1000, 64)])
def test_residual_matches_dot2(n, nrhs):
    A = inputs.gram_shift(n, 1.0, seed=n)
    X = inputs.uniform(n, nrhs, seed=2)
    B = inputs.uniform(n, nrhs, seed=3)
    Ad, _ = to_dev_colmajor(lower_only(A))
    Xd, _ = to_dev_colmajor(X)
    Bd, _ = to_dev_colmajor(B)
    R, cm = jmg.residual(Ad, Xd, Bd)
    Ro = oracle.resid_dot2(A.numpy(), X.numpy(), B.numpy())
    Af = lower_sym_full(A.numpy())
    bound = 2 * n * U64 * (np.abs(Af) @ np.abs(X.numpy()) + np.abs(B.numpy()))
    assert np.all(np.abs(host(R) - Ro) <= bound + 1e-300)
    cm = cm.cpu().numpy()
    assert np.allclose(cm[0], np.abs(host(R)).max(axis=0), rtol=0, atol=0)
    assert np.array_equal(cm[1], np.abs(X.numpy()).max(axis=0))
    assert np.array_equal(cm[2], np.abs(B.numpy()).max(axis=0))


@pytest.mark.parametrize("n", [1, 63, 64, 65, 300])
def test_norm_inf_matches_oracle(n):
    A = inputs.gram_shift(n, 1.0, seed=n + 7)
    A = A - 0.3  # mixed signs
    Ad, _ = to_dev_colmajor(lower_only(A))
    g = float(jmg.norm_inf(Ad).item())
    o = oracle.norm_inf(A.numpy())
    assert abs(g - o) <= 4 * n * U64 * o


@pytest.mark.parametrize("m,ncols", [(1, 1), (100, 100), (128, 128), (129, 129), (300, 300),
                                     (511, 511), (2600, 2600), (4000, 4000), (2600, 700),
                                     (1000, 128)])
@pytest.mark.parametrize("kext", [64, 192])
@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_syrk_tc_exact_integers(m, ncols, kext, dtype):
    # small integers: products and FP32 sums are exact, so the tensor-core
    # update must equal the integer result bit for bit
    g = torch.Generator().manual_seed(m * 1000 + kext)
    PA = torch.randint(-8, 9, (m, kext), generator=g).to(torch.float64)
    PB = torch.randint(-8, 9, (m, kext), generator=g).to(torch.float64)
    C0 = torch.randint(-1000, 1000, (m, m), generator=g).to(torch.float64)
    want = C0 - PA @ PB.t()
    Cd, _ = to_dev_colmajor(C0.to(torch.float32).to(torch.float64))
    Cf = Cd.to(torch.float32)
    Cf = Cf.t().contiguous().t()
    err = jmg.syrk_tc_(Cf, PA.to(DEV).to(dtype).contiguous(), PB.to(DEV).to(dtype).contiguous(),
                       ncols=ncols)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = Cf.double().cpu().numpy()
    w = want.numpy()
    touched = np.tril(np.ones((m, m), dtype=bool))
    touched[:, ncols:] = False
    assert np.array_equal(got[touched], w[touched])
    assert np.array_equal(got[~touched], C0.numpy()[~touched]), "outside the trapezoid was written"


@pytest.mark.parametrize("m,ncols,kext", [(1, 1, 128), (300, 300, 128), (2600, 2600, 128),
                                          (2600, 900, 256)])
def test_syrk_fp8_exact_integers(m, ncols, kext):
    # e4m3 holds the integers -8..8 exactly; products <= 64, sums over kext and
    # power-of-two tile scales stay exact in FP32: the update must be bit-exact
    g = torch.Generator().manual_seed(m + kext)
    Qv = torch.randint(-8, 9, (m, kext), generator=g).to(torch.float64)
    ntile = (m + 127) // 128
    e = torch.randint(-3, 4, (ntile,), generator=g, dtype=torch.int8)
    C0 = torch.randint(-1000, 1000, (m, m), generator=g).to(torch.float64)
    sc = torch.pow(2.0, -e.to(torch.float64))
    rs = sc.repeat_interleave(128)[:m]
    want = C0 - (rs[:, None] * Qv) @ (rs[:, None] * Qv).t()
    Q8 = Qv.to(torch.float32).to(torch.float8_e4m3fn).view(torch.uint8).contiguous().to(DEV)
    Cd, _ = to_dev_colmajor(C0)
    Cf = Cd.to(torch.float32).t().contiguous().t()
    err = jmg.syrk_fp8_(Cf, Q8, e.to(DEV), ncols=ncols)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = Cf.double().cpu().numpy()
    touched = np.tril(np.ones((m, m), dtype=bool))
    touched[:, ncols:] = False
    assert np.array_equal(got[touched], want.numpy()[touched])
    assert np.array_equal(got[~touched], C0.numpy()[~touched])


@pytest.mark.parametrize("m,kext", [(300, 256), (1000, 512), (2600, 1024)])
def test_syrk_fp8_chunk_scales_exact(m, kext):
    # every 128-deep chunk of K has its own power-of-two tile exponents (one
    # panel of the two-level factorisation each); with small integer codes and
    # exponents in [-1, 1] every scaled partial sum needs at most 21 bits, so
    # the FP32 accumulation is exact and the update must be bit-exact
    g = torch.Generator().manual_seed(m * 7 + kext)
    Qv = torch.randint(-8, 9, (m, kext), generator=g).to(torch.float64)
    ntile, nch = (m + 127) // 128, kext // 128
    e = torch.randint(-1, 2, (nch, ntile + 1), generator=g, dtype=torch.int8)
    C0 = torch.randint(-1000, 1000, (m, m), generator=g).to(torch.float64)
    want = C0.clone()
    for c in range(nch):
        rs = torch.pow(2.0, -e[c, :ntile].to(torch.float64)).repeat_interleave(128)[:m]
        Qc = rs[:, None] * Qv[:, 128 * c:128 * (c + 1)]
        want -= Qc @ Qc.t()
    Q8 = Qv.to(torch.float32).to(torch.float8_e4m3fn).view(torch.uint8).contiguous().to(DEV)
    Cd, _ = to_dev_colmajor(C0)
    Cf = Cd.to(torch.float32).t().contiguous().t()
    err = jmg.syrk_fp8_chunks_(Cf, Q8, e.contiguous().to(DEV))
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = Cf.double().cpu().numpy()
    lo = np.tril(np.ones((m, m), dtype=bool))
    assert np.array_equal(got[lo], want.numpy()[lo])
    assert np.array_equal(got[~lo], C0.numpy()[~lo])


def test_syrk_tc_exact_near_fp32_limit():
    # the split residual relies on exact FP32 accumulation of integer products
    # up to ~2^23 in TMEM: all-maximal slices (128 * 128 * 256 = 2^22) and random ones
    m, kext = 256, 256
    for PA in (torch.full((m, kext), 128.0, dtype=torch.float64),
               torch.randint(-128, 129, (m, kext), generator=torch.Generator().manual_seed(5)).double()):
        PB = PA.clone()
        PB[1::2] = torch.clamp(PB[1::2], -64, 64)
        want = -(PA @ PB.t())
        Cf = torch.zeros((m, m), dtype=torch.float32, device=DEV).t().contiguous().t()
        err = jmg.syrk_tc_(Cf, PA.to(DEV).to(torch.bfloat16).contiguous(),
                           PB.to(DEV).to(torch.bfloat16).contiguous())
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        lo = np.tril_indices(m)
        assert np.array_equal(Cf.double().cpu().numpy()[lo], want.numpy()[lo])


@pytest.mark.parametrize("n,nrhs", [(1, 1), (100, 5), (300, 17), (1000, 40), (2100, 64),
                                    (700, 3)])
def test_residual_split_matches_dot2(n, nrhs):
    # FP64-accurate: within the same bound as the CUDA-core FP64 residual
    A = inputs.q_lambda(n, 1e8, seed=n) if n > 1 else inputs.gram_shift(1, 1.0, seed=1)
    X = inputs.uniform(n, nrhs, seed=2)
    B = inputs.rhs_from(A, X) + inputs.uniform(n, nrhs, seed=3) * 1e-6
    Ad, _ = to_dev_colmajor(lower_only(A))
    Xd, _ = to_dev_colmajor(X)
    Bd, _ = to_dev_colmajor(B)
    R, cm, err = jmg.residual_split(Ad, Xd, Bd)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    Ro = oracle.resid_dot2(A.numpy(), X.numpy(), B.numpy())
    Af = lower_sym_full(A.numpy())
    bound = 2 * n * U64 * (np.abs(Af) @ np.abs(X.numpy()) + np.abs(B.numpy()))
    assert np.all(np.abs(host(R) - Ro) <= bound + 1e-300)
    assert np.array_equal(cm.cpu().numpy()[1], np.abs(X.numpy()).max(axis=0))
