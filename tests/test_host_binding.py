"""CPU-only check of the host-buffer binding's marshalling: ``jmg.posv_host``
hands the library the host pointers, leading dimensions, storage type and
options of its arguments, and a device workspace of the size the library asks
for.  The library call itself is replaced by a recorder (no GPU here)."""
from __future__ import annotations

import contextlib

import pytest
import torch

from paper_2601_14466_gb300 import jmg


class _Recorder:
    def __init__(self, real):
        self.real = real
        self.calls = []

    def __getattr__(self, name):
        return getattr(self.real, name)

    def jmg_posv_host(self, *args):
        self.calls.append(args)
        args[9]._obj.value = 0  # the host info word
        return 0


@pytest.fixture
def fake(monkeypatch):
    rec = _Recorder(jmg.load())
    monkeypatch.setattr(jmg, "load", lambda build_if_missing=True: rec)
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "device", lambda d: contextlib.nullcontext())
    monkeypatch.setattr(jmg, "_stream", lambda dev: 1234)
    sizes = []

    def workspace(op, n, nrhs, opts, device, dtype=jmg.JMG_F64):
        nbytes = jmg.workspace_size(op, n, nrhs, opts, dtype)
        sizes.append((op, n, nrhs, dtype, nbytes))
        return torch.empty(max(nbytes, 256), dtype=torch.uint8)  # stands in for device memory

    monkeypatch.setattr(jmg, "workspace", workspace)
    rec.sizes = sizes
    return rec


def test_posv_host_passes_host_pointers_and_strides(fake):
    n, nrhs, lda, ldb = 50, 3, 53, 57
    Abuf = torch.zeros((n, lda), dtype=torch.float64)
    Bbuf = torch.zeros((nrhs, ldb), dtype=torch.float64)
    A, B = Abuf.t()[:n, :], Bbuf.t()[:n, :]
    X, si = jmg.posv_host(A, B, prec="bf16", words=2, nb=64, tol=1e-12, maxit=17)
    (args,) = fake.calls
    (nn, nr, pa, la, pb, lb, px, lx, dt, _info, opts, _stats, pw, lw, stream) = args
    assert (nn, nr, la, lb, lx, dt, stream) == (n, nrhs, lda, ldb, n, jmg.JMG_F64, 1234)
    assert pa == A.data_ptr() and pb == B.data_ptr() and px == X.data_ptr()
    o = opts._obj
    assert (o.prec, o.words, o.nb, o.maxit) == (1, 2, 64, 17) and abs(o.tol - 1e-12) < 1e-25
    assert fake.sizes == [(jmg.OP_POSV_HOST, n, nrhs, jmg.JMG_F64, lw)]
    assert X.shape == (n, nrhs) and X.stride(0) == 1 and not X.is_cuda
    assert si.status == 0 and si.info == 0


def test_posv_host_out_and_float32(fake):
    n = 20
    A = torch.zeros((n, n), dtype=torch.float32).t()
    B = torch.zeros((2, n), dtype=torch.float32).t()
    X, _ = jmg.posv_host(A, B, out=B)
    args = fake.calls[-1]
    assert args[6] == B.data_ptr() and args[8] == jmg.JMG_F32 and X.data_ptr() == B.data_ptr()
    assert fake.sizes[-1][3] == jmg.JMG_F32
    # argument errors are raised before the library is called
    with pytest.raises(TypeError):
        jmg.posv_host(A, B, prec="fp16")
    with pytest.raises(ValueError):
        jmg.posv_host(A, torch.zeros((2, n + 1), dtype=torch.float32).t())
    with pytest.raises(ValueError):
        jmg.posv_host(A, B, out=torch.zeros((3, n), dtype=torch.float32).t())
    with pytest.raises(ValueError):
        jmg.posv_host(A, torch.zeros((n, 2), dtype=torch.float32))  # row-major B
    assert len(fake.calls) == 1


def test_posv_host_refuses_without_a_gpu():
    if torch.cuda.is_available():
        pytest.skip("checks the refusal on a machine without a CUDA device")
    with pytest.raises(RuntimeError):
        jmg.posv_host(torch.eye(3, dtype=torch.float64), torch.ones(3, 1, dtype=torch.float64))
