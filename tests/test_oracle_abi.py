"""CPU test: the oracle's ctypes view of its C structures and functions equals the C source.

oracle/__init__.py restates or_config and or_stats of oracle/dgsrhd_oracle.c as ctypes
structures and gives every exported routine its argument list.  A field or argument changed
on one side only would hand the oracle a shifted configuration and make every parity test
compare against the wrong problem.  A small C program that includes the oracle's source prints
sizeof and offsetof of every field, and the exported routines' parameter lists are read from
the source and compared with the ctypes argument types.
"""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOURCE = os.path.join(ROOT, "oracle", "dgsrhd_oracle.c")

STRUCTS = (("or_config", oracle.Config), ("or_stats", oracle.Stats))


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{SOURCE}"', "int main(void) {"]
    for cname, ctype in STRUCTS:
        lines.append(f'  printf("sizeof {cname} %zu\\n", sizeof({cname}));')
        for field, _ in ctype._fields_:
            lines.append(f'  printf("offset {cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("oracle_abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-D_GNU_SOURCE", str(src), "-o", str(exe), "-lm"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    sizes, offsets = {}, {}
    for line in out.splitlines():
        kind, *rest = line.split()
        if kind == "sizeof":
            sizes[rest[0]] = int(rest[1])
        else:
            offsets[(rest[0], rest[1])] = int(rest[2])
    return sizes, offsets


@pytest.mark.parametrize("cname,ctype", STRUCTS)
def test_struct_layout_matches_the_source(c_layout, cname, ctype):
    sizes, offsets = c_layout
    assert ctypes.sizeof(ctype) == sizes[cname]
    for field, _ in ctype._fields_:
        assert getattr(ctype, field).offset == offsets[(cname, field)], field


def test_struct_fields_are_all_bound():
    """Every member of the two C structures has a ctypes field, in order."""
    text = re.sub(r"/\*.*?\*/", "", open(SOURCE).read(), flags=re.S)
    for cname, ctype in STRUCTS:
        body = re.search(r"typedef struct \{([^{}]*)\} %s;" % cname, text, flags=re.S).group(1)
        declared = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            _, names = decl.split(None, 1)
            declared += [re.match(r"\s*([a-z_0-9]+)", n).group(1) for n in names.split(",")]
        assert declared == [f for f, _ in ctype._fields_], cname


SCALARS = {"int": ctypes.c_int, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
           "double": ctypes.c_double}
POINTEES = dict(SCALARS, or_config=oracle.Config, or_stats=oracle.Stats)


def test_routine_arguments_match_the_source():
    lib = oracle._load()
    text = re.sub(r"/\*.*?\*/", "", open(SOURCE).read(), flags=re.S)
    defs = re.findall(r"^(int|double|void)\s+(or_[a-z_0-9]+)\s*\(([^)]*)\)\s*\{", text, flags=re.M)
    bound = 0
    for ret, name, params in defs:
        fn = getattr(lib, name)
        if fn.argtypes is None:
            continue  # exported but not called from Python
        bound += 1
        types = [" ".join(p.split()) for p in params.split(",") if p.strip() not in ("", "void")]
        assert len(fn.argtypes) == len(types), name
        for k, (ct, pt) in enumerate(zip(fn.argtypes, types)):
            pt = re.sub(r"\s*\b[a-zA-Z_][a-zA-Z_0-9]*$", "", pt).replace("const ", "").replace(" *", "*")
            where = f"{name} argument {k}"
            if pt.endswith("*"):
                assert issubclass(ct, ctypes._Pointer) and ct._type_ is POINTEES[pt[:-1].strip()], where
            else:
                assert ct is SCALARS[pt], where
        want_res = {"int": ctypes.c_int, "double": ctypes.c_double, "void": None}[ret]
        assert fn.restype is want_res, name
    assert bound >= 15, "the ctypes bindings were not found"
