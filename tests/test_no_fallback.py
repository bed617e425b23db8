"""The product path has no fallback: without its CUDA library the package raises,
and no file of the package imports, loads or links the oracle."""
import os
import re

import numpy as np
import pytest

import paper_1908_05944_gb300 as ac

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1908_05944_gb300")


def test_missing_library_raises(monkeypatch):
    monkeypatch.setattr(ac, "_lib", None)
    monkeypatch.setattr(ac, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libalphac.so"))
    with pytest.raises(RuntimeError, match="not built"):
        ac.lib()
    with pytest.raises(RuntimeError, match="not built"):
        ac.AlphaComplex(np.zeros((1, 3)), np.ones(1), 0.0)
    with pytest.raises(RuntimeError, match="not built"):
        ac.chunk_plan(np.zeros((1, 3)), np.ones(1), 0.0)


def test_package_never_touches_the_oracle():
    pattern = re.compile(r"\boracle\b|alpha_oracle|liboracle")
    offenders = []
    for dirpath, dirnames, filenames in os.walk(PKG):
        dirnames[:] = [d for d in dirnames if d not in ("_build", "__pycache__")]
        for name in filenames:
            if not name.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                continue
            path = os.path.join(dirpath, name)
            for k, line in enumerate(open(path, encoding="utf-8"), 1):
                if pattern.search(line):
                    offenders.append(f"{os.path.relpath(path, ROOT)}:{k}: {line.strip()}")
    assert not offenders, "the package refers to the oracle:\n" + "\n".join(offenders)


def test_oracle_shares_no_code_with_the_package():
    # the oracle includes only the C standard library and imports nothing of the package
    src = open(os.path.join(ROOT, "oracle", "alpha_oracle.c"), encoding="utf-8").read()
    includes = re.findall(r'#include\s*[<"]([^>"]+)[>"]', src)
    assert includes and all(i in ("math.h", "pthread.h", "stdint.h", "stdlib.h", "string.h") for i in includes)
    py = open(os.path.join(ROOT, "oracle", "__init__.py"), encoding="utf-8").read()
    assert not re.search(r"^\s*(import|from)\s+(paper_1908_05944_gb300|synth)\b", py, re.M)
