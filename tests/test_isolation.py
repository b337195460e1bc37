"""CPU-only checks that the product path and the oracle stay apart.

The library and its binding must neither import, include nor link anything of
the oracle (the oracle is test infrastructure), the oracle must not use the
library, and the binding must refuse to run when the CUDA library is absent
instead of falling back to some other implementation.
"""
from __future__ import annotations

import glob
import os
import re

import pytest

from paper_2601_14466_gb300 import _build, jmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2601_14466_gb300")


def _strip_comments(text: str, lang: str) -> str:
    if lang == "c":
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        return re.sub(r"//[^\n]*", "", text)
    text = re.sub(r'""".*?"""', "", text, flags=re.S)
    return re.sub(r"#[^\n]*", "", text)


def _package_sources():
    py = glob.glob(os.path.join(PKG, "*.py"))
    c = (glob.glob(os.path.join(PKG, "csrc", "*.cu")) + glob.glob(os.path.join(PKG, "csrc", "*.h"))
         + glob.glob(os.path.join(PKG, "csrc", "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h")))
    return [(p, "py") for p in py] + [(p, "c") for p in c]


def test_package_never_touches_the_oracle():
    bad = []
    for path, lang in _package_sources():
        code = _strip_comments(open(path).read(), lang)
        if lang == "py":
            if re.search(r"^\s*(import\s+oracle|from\s+oracle\b)", code, flags=re.M) or \
                    re.search(r"\boracle\b", code):
                bad.append(path)
        elif re.search(r"oracle", code):
            bad.append(path)
    assert not bad, bad
    # and the library's link line names no oracle object or library
    assert not any("oracle" in f for f in _build.NVCC_FLAGS)


def test_oracle_never_touches_the_package():
    code_c = _strip_comments(open(os.path.join(ROOT, "oracle", "oracle.c")).read(), "c")
    assert "jmg" not in code_c and "#include \"" not in code_c
    code_py = _strip_comments(open(os.path.join(ROOT, "oracle", "__init__.py")).read(), "py")
    assert "paper_2601_14466_gb300" not in code_py and "libjmg" not in code_py


def test_input_generators_hold_no_solver_call():
    # the seeded generators serve both sides, so they may not reach either one
    code = _strip_comments(open(os.path.join(PKG, "inputs.py")).read(), "py")
    for word in ("jmg", "oracle", "cholesky", "solve", "ctypes"):
        assert word not in code.lower(), word


def test_missing_library_raises_instead_of_falling_back(monkeypatch, tmp_path):
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "absent" / "libjmg.so"))
    monkeypatch.setattr(jmg, "_lib", None)
    with pytest.raises(RuntimeError):
        jmg.load(build_if_missing=False)
