"""posv on HOST buffers (``jmg_posv_host``) against the oracle: the call copies
lower(A) and B to the device, solves there and copies X back.  Checked: the
solution (oracle backward error and forward error, as for the device-buffer
call), the host inputs left untouched, the copy volumes it reports, padding
and NaN canaries outside lower(A), aliasing X with B, page-locked and pageable
buffers, FP32 storage, and the non-SPD report.  Paper: "Software design"
(potrs semantics)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2601_14466_gb300 import inputs, jmg
from tests.helpers import U64, lower_only

pytestmark = pytest.mark.gpu

def host_colmajor(M: torch.Tensor, lda: int | None = None, fill=float("nan"), pinned=False,
                  dtype=torch.float64):
    """Column-major host copy with leading dimension lda (padding rows = fill)."""
    n, m = M.shape
    lda = lda or n
    buf = torch.full((m, lda), fill, dtype=dtype, pin_memory=pinned)
    view = buf.t()
    view[:n, :].copy_(M.to(dtype))
    return view[:n, :], buf


def expected_h2d(n, nrhs, es):
    return es * (n * n + n * nrhs)  # the n x n block of A, then B


def same(a: torch.Tensor, b: torch.Tensor) -> bool:
    return torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("n,nrhs,pad", [(1, 1, 0), (100, 5, 3), (257, 2, 0), (700, 64, 1),
                                        (1300, 17, 0)])
def test_posv_host_fp64_matches_oracle(n, nrhs, pad, pinned):
    kappa = 1e3
    A = inputs.q_lambda(n, kappa, seed=inputs.seed_for("host", n))
    Xt = inputs.uniform(n, nrhs, seed=3)
    B = inputs.rhs_from(A, Xt)
    Ah, Abuf = host_colmajor(lower_only(A), lda=n + pad, pinned=pinned)
    Bh, Bbuf = host_colmajor(B, lda=n + pad, pinned=pinned)
    A0, B0 = Abuf.clone(), Bbuf.clone()
    X, si = jmg.posv_host(Ah, Bh, prec="fp64")
    assert not X.is_cuda and X.shape == (n, nrhs) and X.stride(0) == 1
    assert si.status == 0 and si.info == 0
    Xg = np.asfortranarray(X.numpy())
    eta, _ = oracle.bwd_err(A.numpy(), Xg, B.numpy())
    assert eta <= 1e-13, eta
    Xo, _ = oracle.posv(A.numpy(), B.numpy())
    assert np.abs(Xg - Xo).max() <= 100 * kappa * n * U64 * np.abs(Xo).max()
    # the host inputs, canaries and padding included, are untouched
    assert same(Abuf, A0) and same(Bbuf, B0)
    # A (n x n, padding rows skipped) and B in, X back
    assert si.h2d_bytes == expected_h2d(n, nrhs, 8)
    assert si.d2h_bytes == 8 * n * nrhs


@pytest.mark.parametrize("prec,words,nb", [("fp16", 2, 128), ("bf16", 2, 64), ("bf16", 1, 128)])
@pytest.mark.parametrize("n,nrhs", [(130, 1), (1100, 16)])
def test_posv_host_mixed_matches_oracle(prec, words, nb, n, nrhs):
    A = inputs.gram_shift(n, 1.0, seed=inputs.seed_for("hostmix", n))
    Xt = inputs.uniform(n, nrhs, seed=4)
    B = inputs.rhs_from(A, Xt)
    Ah, Abuf = host_colmajor(lower_only(A), pinned=True)
    Bh, _ = host_colmajor(B, pinned=True)
    A0 = Abuf.clone()
    X, si = jmg.posv_host(Ah, Bh, prec=prec, words=words, nb=nb)
    assert si.status == 0 and si.info == 0 and si.bwd_err <= 1e-13
    assert si.iters >= 1 and si.factor_tries >= 1
    Xg = np.asfortranarray(X.numpy())
    eta, _ = oracle.bwd_err(A.numpy(), Xg, B.numpy())
    assert eta <= 1e-13, eta
    Xo, _ = oracle.posv(A.numpy(), B.numpy())
    assert np.abs(Xg - Xo).max() <= 4 * 10.0 * 1e-13 * np.abs(Xo).max() * 10
    assert same(Abuf, A0)
    assert si.h2d_bytes == expected_h2d(n, nrhs, 8) and si.d2h_bytes == 8 * n * nrhs


def test_posv_host_out_may_alias_b_and_vectors():
    n = 600
    A = inputs.gram_shift(n, 1.0, seed=11)
    B = inputs.uniform(n, 3, seed=12)
    Ah, _ = host_colmajor(A, pinned=True)
    Bh, _ = host_colmajor(B, pinned=True)
    X, si = jmg.posv_host(Ah, Bh, prec="bf16", words=2, out=Bh)
    assert X.data_ptr() == Bh.data_ptr() and si.status == 0
    Xo, _ = oracle.posv(A.numpy(), B.numpy())
    assert np.abs(np.asfortranarray(Bh.numpy()) - Xo).max() <= 1e-11 * np.abs(Xo).max()
    # one right-hand side as a 1-D tensor comes back 1-D
    b = B[:, 0].contiguous()
    x, si = jmg.posv_host(Ah, b, prec="fp64")
    assert x.dim() == 1 and si.status == 0
    assert np.abs(x.numpy() - Xo[:, 0]).max() <= 1e-11 * np.abs(Xo).max()


def test_posv_host_fp32_storage():
    n, nrhs = 400, 6
    A = inputs.gram_shift(n, 1.0, seed=13).to(torch.float32).to(torch.float64)
    A = 0.5 * (A + A.t())
    B = inputs.uniform(n, nrhs, seed=14).to(torch.float32).to(torch.float64)
    Ah, _ = host_colmajor(lower_only(A), dtype=torch.float32, pinned=True)
    Bh, _ = host_colmajor(B, dtype=torch.float32, pinned=True)
    X, si = jmg.posv_host(Ah, Bh, prec="fp64")
    assert X.dtype == torch.float32 and si.status == 0
    eta, _ = oracle.bwd_err(A.numpy(), np.asfortranarray(X.to(torch.float64).numpy()), B.numpy())
    assert eta <= 8 * n * 2.0 ** -24
    assert si.h2d_bytes == expected_h2d(n, nrhs, 4) and si.d2h_bytes == 4 * n * nrhs
    with pytest.raises(TypeError):
        jmg.posv_host(Ah, Bh, prec="bf16")


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_posv_host_not_spd(prec):
    n = 300
    A = inputs.gram_shift(n, 1.0, seed=2)
    A[100, 100] = -50.0
    Ah, _ = host_colmajor(A, pinned=True)
    Bh, _ = host_colmajor(inputs.uniform(n, 1, seed=1), pinned=True)
    _, si = jmg.posv_host(Ah, Bh, prec=prec, shift_retry=False, check=False)
    assert si.status == 3 and si.info == 101  # JMG_ERR_NOT_SPD, leading minor 101
    with pytest.raises(jmg.JmgError):
        jmg.posv_host(Ah, Bh, prec=prec, shift_retry=False)


def test_posv_host_rejects_device_tensors_and_empty_is_a_no_op():
    A = torch.eye(4, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        jmg.posv_host(A, torch.ones(4, 1, dtype=torch.float64))
    X, si = jmg.posv_host(torch.zeros(0, 0, dtype=torch.float64),
                          torch.zeros(2, 0, dtype=torch.float64).t())
    assert X.shape == (0, 2) and si.status == 0 and si.info == 0
