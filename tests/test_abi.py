"""CPU-only checks of the C ABI: the library builds and loads, exports every
symbol that include/*.h declares, and rejects illegal arguments (LAPACK-style
negative codes) before touching the GPU."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

from paper_2601_14466_gb300 import jmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(jmg_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_the_core_calls():
    d = declared_symbols()
    for name in ("jmg_potrf", "jmg_potrs", "jmg_posv", "jmg_workspace_size", "jmg_logdet"):
        assert name in d


def test_library_exports_every_declared_symbol():
    lib = jmg.load()
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    # and the binding wires every one of them
    assert set(declared_symbols()) <= set(jmg.exported_symbols())


def test_illegal_arguments_are_rejected_on_the_host():
    lib = jmg.load()
    info = ctypes.c_void_p(1)  # never dereferenced: the checks fire first
    assert lib.jmg_potrf(-1, None, 1, 0, info, None, None, 0, None) == -1
    assert lib.jmg_potrf(10, None, 5, 0, info, None, None, 0, None) == -3
    assert lib.jmg_potrf(10, None, 10, 9, info, None, None, 0, None) == -4
    assert lib.jmg_potrf(10, None, 10, 0, None, None, None, 0, None) == -5
    assert lib.jmg_potrs(-1, 1, None, 1, None, 1, 0, None, 0, None) == -1
    assert lib.jmg_potrs(4, -1, None, 4, None, 4, 0, None, 0, None) == -2
    assert lib.jmg_potrs(4, 1, None, 3, None, 4, 0, None, 0, None) == -4
    assert lib.jmg_potrs(4, 1, None, 4, None, 3, 0, None, 0, None) == -6
    assert lib.jmg_potrs(0, 0, None, 1, None, 1, 0, None, 0, None) == 0
    assert lib.jmg_posv(-2, 1, None, 1, None, 1, 0, info, None, None, None, 0, None) == -1
    assert lib.jmg_posv(4, 1, None, 4, None, 4, 0, None, None, None, None, 0, None) == -8
    o = jmg.default_options(nb=100)
    assert lib.jmg_posv(4, 1, None, 4, None, 4, 0, info, ctypes.byref(o), None, None, 0,
                        None) == -9
    # mixed posv without workspace
    o = jmg.default_options(prec="bf16")
    assert lib.jmg_posv(256, 2, ctypes.c_void_p(256), 256, ctypes.c_void_p(512), 256, 0, info,
                        ctypes.byref(o), None, None, 0, None) == 2  # JMG_ERR_WORKSPACE


def test_defaults_and_workspace():
    o = jmg.default_options()
    assert (o.nb, o.prec, o.words, o.maxit, o.reuse_factor) == (128, 0, 1, 300, 0)
    assert abs(o.tol - 1e-13) < 1e-30
    assert jmg.workspace_size(jmg.OP_POTRF, 1000, 1, o) == 0
    # the plain solves only need their tickets and flags
    assert 0 < jmg.workspace_size(jmg.OP_POSV, 1000, 4, o) <= 4096
    assert 0 < jmg.workspace_size(jmg.OP_POTRS, 1000, 4, o) <= 4096
    assert jmg.workspace_size(jmg.OP_POTRS, 0, 4, o) == 0
    om = jmg.default_options(prec="bf16")
    w1 = jmg.workspace_size(jmg.OP_POSV, 1000, 4, om)
    w2 = jmg.workspace_size(jmg.OP_POSV, 2000, 4, om)
    assert 4 * 1000 * 1000 <= w1 < w2
    om3 = jmg.default_options(prec="bf16", words=3)
    assert jmg.workspace_size(jmg.OP_POSV, 1000, 4, om3) > w1
    assert jmg.load().jmg_status_string(3) == b"matrix is not positive definite"


def test_no_cpu_fallback():
    import torch

    if torch.cuda.is_available():
        pytest.skip("checks the CPU-only refusal")
    A = torch.eye(4, dtype=torch.float64)
    with pytest.raises(ValueError):
        jmg.posv(A, torch.ones(4, 1, dtype=torch.float64))


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of jmg_options / jmg_stats must have the C layout
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "jmg.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu %zu %zu %zu\\n", '
                   'sizeof(jmg_options), sizeof(jmg_stats), offsetof(jmg_stats, eta_hist), '
                   'offsetof(jmg_stats, n_solve), offsetof(jmg_stats, t_factor_gpu_ms), '
                   'offsetof(jmg_stats, h2d_bytes), offsetof(jmg_stats, d2h_bytes)); '
                   'return 0; }\n')
    exe = tmp_path / "sizes"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    want = [ctypes.sizeof(jmg.Options), ctypes.sizeof(jmg.Stats), jmg.Stats.eta_hist.offset,
            jmg.Stats.n_solve.offset, jmg.Stats.t_factor_gpu_ms.offset,
            jmg.Stats.h2d_bytes.offset, jmg.Stats.d2h_bytes.offset]
    assert got == want


def test_posv_batched_argument_checks():
    lib = jmg.load()
    f = lib.jmg_posv_batched
    # (n, nrhs, batch, A, lda, sA, B, ldb, sB, dtype, info, stream)
    assert f(-1, 1, 1, 256, 1, 1, 256, 1, 1, jmg.JMG_F64, 256, None) == -1
    assert f(4, -1, 1, 256, 4, 16, 256, 4, 4, jmg.JMG_F64, 256, None) == -2
    assert f(4, 1, -1, 256, 4, 16, 256, 4, 4, jmg.JMG_F64, 256, None) == -3
    assert f(4, 1, 1, 256, 3, 16, 256, 4, 4, jmg.JMG_F64, 256, None) == -5
    assert f(4, 1, 1, 256, 4, 15, 256, 4, 4, jmg.JMG_F64, 256, None) == -6
    assert f(4, 1, 1, 256, 4, 16, 256, 3, 4, jmg.JMG_F64, 256, None) == -8
    assert f(4, 2, 1, 256, 4, 16, 256, 4, 4, jmg.JMG_F64, 256, None) == -9
    assert f(4, 1, 1, 256, 4, 16, 256, 4, 4, 9, 256, None) == -10
    assert f(4, 1, 1, 256, 4, 16, 256, 4, 4, jmg.JMG_F64, None, None) == -11
    assert f(129, 1, 1, 256, 129, 129 * 129, 256, 129, 129, jmg.JMG_F64, 256, None) == 6


def test_posv_host_argument_checks():
    lib = jmg.load()
    f = lib.jmg_posv_host
    info = ctypes.c_int(-7)
    h = ctypes.c_void_p(4096)  # never dereferenced: the checks fire first
    # (n, nrhs, A, lda, B, ldb, X, ldx, dtype, info, opt, stats, work, lwork, stream)
    assert f(-1, 1, h, 1, h, 1, h, 1, jmg.JMG_F64, ctypes.byref(info), None, None, None, 0,
             None) == -1
    assert f(4, -1, h, 4, h, 4, h, 4, jmg.JMG_F64, ctypes.byref(info), None, None, None, 0,
             None) == -2
    assert f(4, 1, h, 3, h, 4, h, 4, jmg.JMG_F64, ctypes.byref(info), None, None, None, 0,
             None) == -4
    assert f(4, 1, h, 4, h, 3, h, 4, jmg.JMG_F64, ctypes.byref(info), None, None, None, 0,
             None) == -6
    assert f(4, 1, h, 4, h, 4, h, 3, jmg.JMG_F64, ctypes.byref(info), None, None, None, 0,
             None) == -8
    assert f(4, 1, h, 4, h, 4, h, 4, 5, ctypes.byref(info), None, None, None, 0, None) == -9
    assert f(4, 1, h, 4, h, 4, h, 4, jmg.JMG_F64, None, None, None, None, 0, None) == -10
    o = jmg.default_options(nb=96)
    assert f(4, 1, h, 4, h, 4, h, 4, jmg.JMG_F64, ctypes.byref(info), ctypes.byref(o), None,
             None, 0, None) == -11
    o = jmg.default_options(prec="fp8", nb=64)
    assert f(4, 1, h, 4, h, 4, h, 4, jmg.JMG_F64, ctypes.byref(info), ctypes.byref(o), None,
             None, 0, None) == -11
    # n == 0: nothing to do, info cleared, no device touched
    assert f(0, 3, None, 1, None, 1, None, 1, jmg.JMG_F64, ctypes.byref(info), None, None,
             None, 0, None) == 0 and info.value == 0
    assert f(4, 1, None, 4, h, 4, h, 4, jmg.JMG_F64, ctypes.byref(info), None, None, None, 0,
             None) == -3
    assert f(4, 1, h, 4, None, 4, h, 4, jmg.JMG_F64, ctypes.byref(info), None, None, None, 0,
             None) == -5
    assert f(4, 1, h, 4, h, 4, None, 4, jmg.JMG_F64, ctypes.byref(info), None, None, None, 0,
             None) == -7
    # mixed modes refine FP64 data only
    o = jmg.default_options(prec="bf16")
    assert f(4, 1, h, 4, h, 4, h, 4, jmg.JMG_F32, ctypes.byref(info), ctypes.byref(o), None,
             None, 0, None) == 6  # JMG_ERR_UNSUPPORTED
    # the staging buffers must fit: checked before any copy is queued
    assert f(4, 1, h, 4, h, 4, h, 4, jmg.JMG_F64, ctypes.byref(info), None, None, None, 0,
             None) == 2  # JMG_ERR_WORKSPACE
    need = jmg.workspace_size(jmg.OP_POSV_HOST, 4, 1)
    assert f(4, 1, h, 4, h, 4, h, 4, jmg.JMG_F64, ctypes.byref(info), None, None,
             ctypes.c_void_p(4096 + 16), need, None) == 7  # JMG_ERR_ALIGN


def test_posv_host_workspace_stages_a_and_b():
    for prec, words in (("fp64", 1), ("bf16", 2), ("fp8", 1)):
        o = jmg.default_options(prec=prec, words=words)
        for n, nrhs in ((1, 1), (257, 3), (4096, 64)):
            for dt, es in ((jmg.JMG_F64, 8), (jmg.JMG_F32, 4)):
                if dt == jmg.JMG_F32 and prec != "fp64":
                    continue
                inner = jmg.workspace_size(jmg.OP_POSV, n, nrhs, o, dt)
                host = jmg.workspace_size(jmg.OP_POSV_HOST, n, nrhs, o, dt)
                stage = host - inner
                # the device copies of A (n x n) and B (n x nrhs), each rounded to
                # 256 bytes, and one 256-byte slot for the device info word
                r = lambda b: (b + 255) // 256 * 256
                assert stage == r(es * n * n) + r(es * n * nrhs) + 256
    assert jmg.workspace_size(jmg.OP_POSV_HOST, 0, 4) == 0
    assert jmg.workspace_size(jmg.OP_POSV_HOST, 10, 4, None, 7) == 0


def test_plain_c_caller_links_and_runs(tmp_path):
    # the headers compile as C11 and a C program linked against libjmg.so runs
    # the host-side checks of the ABI (no GPU needed)
    import subprocess

    lib = jmg.load()
    libdir = os.path.dirname(jmg.lib_path())
    exe = tmp_path / "abi_from_c"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_from_c.c"), "-o", str(exe),
                    "-L" + libdir, "-ljmg", "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
    assert lib is not None
