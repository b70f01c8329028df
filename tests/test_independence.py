"""The oracle and the CUDA path share no code, and the product path cannot
fall back to the oracle (CPU only).

- No Python module of the package imports the oracle, and no oracle module
  imports the package; the only code both sides use is the input generator
  (`synth`), which holds none of the method's arithmetic.
- The oracle's C source includes only the C standard library and pthreads;
  no CUDA source includes anything from `oracle/`.
- The binding raises when the CUDA library is missing instead of computing
  anything itself."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_0902_0915_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def _py_files(d):
    for base, _, files in os.walk(d):
        if "__pycache__" in base or "_lib" in base:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_package_never_imports_the_oracle():
    for f in _py_files(PKG):
        assert "oracle" not in _imports(f), f


def test_oracle_never_imports_the_package():
    for f in _py_files(os.path.join(ROOT, "oracle")):
        assert not {"paper_0902_0915_gb300"} & _imports(f), f


def test_generator_holds_no_method_code():
    for f in _py_files(os.path.join(ROOT, "synth")):
        assert not {"paper_0902_0915_gb300", "oracle"} & _imports(f), f


def test_c_sources_stay_apart():
    src = open(os.path.join(ROOT, "oracle", "mwax_oracle.c")).read()
    incs = re.findall(r'#include\s*[<"]([^>"]+)[>"]', src)
    assert set(incs) <= {"pthread.h", "stdint.h", "stdlib.h", "string.h", "math.h", "stdio.h"}, incs
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        for inc in re.findall(r'#include\s*"([^"]+)"', text):
            assert "oracle" not in inc, (f, inc)


def test_missing_library_fails_loudly(monkeypatch):
    import paper_0902_0915_gb300 as mw

    monkeypatch.setattr(mw, "_lib", None)
    monkeypatch.setattr(mw, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libmwax.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        mw.lib()
