"""The FP8 quantiser of the mixed factorisation on its own (the panel of the
factor becomes e4m3 codes with one power-of-two scale per 128-row tile).

Checked against a plain PyTorch restatement of the same op on the CPU: the
tile exponent is e = floor(log2(448 / amax)) clamped to [-126, 126] (0 for an
all-zero tile), every code is round-to-nearest-even of x * 2^e in e4m3 (448 is
the largest finite value, so nothing saturates), and q * 2^-e recovers x
within half an e4m3 ulp.  The codes must agree bit for bit."""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

from paper_2601_14466_gb300 import jmg
from tests.helpers import DEV

pytestmark = pytest.mark.gpu


def _reference(L21: torch.Tensor):
    m, kb = L21.shape
    Q = torch.empty((m, kb), dtype=torch.uint8)
    es = []
    for t0 in range(0, m, 128):
        tile = L21[t0:t0 + 128].double()
        amax = float(tile.abs().max())
        if amax > 0 and math.isfinite(amax):
            e = math.floor(math.log2(448.0 / amax))
            while e > -126 and math.ldexp(amax, e) > 448.0:
                e -= 1
            e = max(-126, min(126, e))
        else:
            e = 0
        es.append(e)
        scaled = (tile * (2.0 ** e)).to(torch.float32)  # exact: a power of two
        Q[t0:t0 + 128] = scaled.to(torch.float8_e4m3fn).view(torch.uint8)
    return Q, torch.tensor(es, dtype=torch.int8)


@pytest.mark.parametrize("m,kb,scale", [(128, 128, 1.0), (300, 128, 1e-3), (1000, 64, 37.0),
                                        (129, 128, 2.0 ** -20)])
def test_quant_fp8_matches_reference(m, kb, scale):
    g = torch.Generator().manual_seed(m + kb)
    L = (torch.randn((m, kb), generator=g, dtype=torch.float64) * scale).to(torch.float32)
    # tiles with very different magnitudes, one exact zero tile when m allows
    L[: min(m, 128)] *= 16.0
    if m >= 256:
        L[128:256] = 0.0
    Ld = L.to(DEV).t().contiguous().t()  # column-major, as the factor stores it
    Q, e = jmg.quant_fp8(Ld)
    torch.cuda.synchronize()
    Qr, er = _reference(L)
    assert torch.equal(e.cpu(), er)
    assert torch.equal(Q.cpu(), Qr)
    # every exponent makes the tile's maximum land in [224, 448]
    for t, t0 in enumerate(range(0, m, 128)):
        amax = float(L[t0:t0 + 128].abs().max())
        if amax > 0:
            assert 224.0 <= math.ldexp(amax, int(er[t])) <= 448.0
    # dequantised codes are within half an e4m3 ulp (relative 2^-4) of x, or
    # below the smallest normal (absolute 2^-10 of the scaled value)
    deq = Q.cpu().view(torch.float8_e4m3fn).to(torch.float64)
    scl = torch.pow(2.0, -er.to(torch.float64)).repeat_interleave(128)[:m, None]
    err = (deq * scl - L.double()).abs()
    bound = torch.maximum(L.double().abs() * 2.0 ** -4, scl * 2.0 ** -10)
    assert bool((err <= bound).all())


def test_quant_fp8_ties_round_to_even():
    # values exactly halfway between two e4m3 codes (after scaling) must go to
    # the even code: 1 + 1/16 -> 1, 1 + 3/16 -> 1.25, 17 -> 16, 19 -> 20
    m, kb = 128, 128
    L = torch.zeros((m, kb), dtype=torch.float32)
    L[0, 0] = 448.0  # fixes e = 0
    vals = [1.0625, 1.1875, 17.0, 19.0, -1.0625, -19.0]
    for k, v in enumerate(vals):
        L[1 + k, 0] = v
    Q, e = jmg.quant_fp8(L.to(DEV).t().contiguous().t())
    torch.cuda.synchronize()
    assert int(e[0]) == 0
    got = Q.cpu().view(torch.float8_e4m3fn).to(torch.float32)[1:1 + len(vals), 0].tolist()
    assert got == [1.0, 1.25, 16.0, 20.0, -1.0, -20.0]
