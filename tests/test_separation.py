"""The oracle and the CUDA path share no code, on CPU: no product file imports, includes or loads
the oracle; the oracle neither imports the package nor includes anything but the C standard
library; bench.py touches the oracle only in its CPU-baseline and reference legs; the shared
input module imports neither side; and the product fails loudly without its CUDA library."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2205_00095_gb300"


def _files(folder, exts):
    for dirpath, dirnames, filenames in os.walk(os.path.join(ROOT, folder)):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_build", "__pycache__"))]
        for f in filenames:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def _imports(path):
    """(module name, enclosing function name or None) of every import in a Python file."""
    tree = ast.parse(open(path).read())
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.Import):
                out.extend((a.name, name) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                out.append(("." * child.level + (child.module or ""), name))
            visit(child, name)

    visit(tree, None)
    return out


def _is(mod, top):
    return mod == top or mod.startswith(top + ".")


def test_product_python_never_imports_the_oracle():
    files = list(_files(PKG, (".py",))) + list(_files("workloads", (".py",)))
    assert files
    for f in files:
        for mod, _ in _imports(f):
            assert not _is(mod, "oracle") and not _is(mod, "tests"), (f, mod)


def test_product_cuda_sources_include_nothing_of_the_oracle():
    files = list(_files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h"))) + \
        list(_files("include", (".h",)))
    assert files
    for f in files:
        text = open(f).read()
        for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', text):
            assert "oracle" not in inc, (f, inc)
        assert "liboracle" not in text and "dgsrhd_oracle" not in text, f


def test_oracle_stands_alone():
    for f in _files("oracle", (".py",)):
        for mod, _ in _imports(f):
            assert not _is(mod, PKG) and not _is(mod, "bench") and not _is(mod, "tests"), (f, mod)
    src = open(os.path.join(ROOT, "oracle", "dgsrhd_oracle.c")).read()
    quoted = re.findall(r'#\s*include\s*"([^"]+)"', src)
    assert quoted == [], quoted
    for inc in re.findall(r'#\s*include\s*<([^>]+)>', src):
        assert inc in {"math.h", "stdlib.h", "string.h", "stdint.h", "stdio.h", "float.h",
                       "stddef.h", "complex.h", "limits.h", "stdbool.h"}, inc


def test_inputs_module_imports_neither_side():
    for f in _files("workloads", (".py",)):
        for mod, _ in _imports(f):
            assert not _is(mod, PKG) and not _is(mod, "oracle"), (f, mod)


def test_bench_uses_the_oracle_only_in_its_cpu_legs():
    legs = {"oracle_sample_spec", "run_oracle"}
    uses = [(m, fn) for m, fn in _imports(os.path.join(ROOT, "bench.py")) if _is(m, "oracle")]
    assert uses and all(fn in legs for _, fn in uses), uses


def test_product_fails_loudly_without_its_cuda_library(monkeypatch, tmp_path):
    from paper_2205_00095_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libdgsrhd.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load()
