"""CPU test: the Python binding's view of the C ABI equals the header's.

The ctypes structures in paper_2205_00095_gb300/_lib.py restate dgsrhd_config and
dgsrhd_stats, and the binding restates the header's status, EOS, solver, flux, boundary, node,
limiter and precision codes.  A field added, reordered or retyped on one side only would pass
every other host test and hand the kernels a shifted configuration.  So a small C program
compiled against include/dgsrhd.h prints sizeof, offsetof and every DGSRHD_* constant, and the
test compares them with the binding.
"""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2205_00095_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dgsrhd.h")


def header_constants():
    text = open(HEADER).read()
    return re.findall(r"^#define\s+(DGSRHD_[A-Z0-9_]+)\s+\S", text, flags=re.M)


def struct_fields(ctype):
    return [name for name, _ in ctype._fields_]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dgsrhd.h"', "int main(void) {"]
    for st in ("dgsrhd_config", "dgsrhd_stats"):
        lines.append(f'  printf("sizeof {st} %zu\\n", sizeof({st}));')
    for name in struct_fields(_lib.dgsrhd_config):
        lines.append(f'  printf("offset dgsrhd_config {name} %zu\\n", offsetof(dgsrhd_config, {name}));')
    for name in struct_fields(_lib.dgsrhd_stats):
        lines.append(f'  printf("offset dgsrhd_stats {name} %zu\\n", offsetof(dgsrhd_stats, {name}));')
    for const in header_constants():
        if const == "DGSRHD_H":
            continue
        lines.append(f'  printf("const {const} %lld\\n", (long long)({const}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HEADER),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    sizes, offsets, consts = {}, {}, {}
    for line in out.splitlines():
        kind, *rest = line.split()
        if kind == "sizeof":
            sizes[rest[0]] = int(rest[1])
        elif kind == "offset":
            offsets[(rest[0], rest[1])] = int(rest[2])
        else:
            consts[rest[0]] = int(rest[1])
    return sizes, offsets, consts


@pytest.mark.parametrize("ctype", [_lib.dgsrhd_config, _lib.dgsrhd_stats])
def test_struct_layout_matches_the_header(c_layout, ctype):
    sizes, offsets, _ = c_layout
    name = ctype.__name__
    assert ctypes.sizeof(ctype) == sizes[name]
    for field in struct_fields(ctype):
        assert getattr(ctype, field).offset == offsets[(name, field)], field


def test_header_struct_fields_are_all_bound():
    """Every member the header declares in the two structures has a ctypes field (the C
    program above would not compile for a ctypes field the header lacks)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for ctype in (_lib.dgsrhd_config, _lib.dgsrhd_stats):
        body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (ctype.__name__, ctype.__name__),
                         text, flags=re.S).group(1)
        declared = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            # "double lo[3], hi[3]" declares two members
            _, names = decl.split(None, 1)
            declared += [re.match(r"\s*([a-z_0-9]+)", n).group(1) for n in names.split(",")]
        assert declared == struct_fields(ctype)


def test_binding_codes_match_the_header(c_layout):
    _, _, c = c_layout
    status = {n: getattr(_lib, n) for n in dir(_lib) if n.startswith("DGSRHD_")}
    assert status, "the binding names no status codes"
    for name, value in status.items():
        assert c[name] == value, name
    groups = {
        "EOS": {"ideal": "DGSRHD_EOS_IDEAL", "tm": "DGSRHD_EOS_TAUB_MATTHEWS",
                "taub_matthews": "DGSRHD_EOS_TAUB_MATTHEWS"},
        "C2P": {"analytic": "DGSRHD_C2P_ANALYTIC", "iterative": "DGSRHD_C2P_ITERATIVE",
                "default": "DGSRHD_C2P_DEFAULT"},
        "FLUX": {"llf": "DGSRHD_FLUX_LLF", "hll": "DGSRHD_FLUX_HLL", "hllc": "DGSRHD_FLUX_HLLC"},
        "BC": {"periodic": "DGSRHD_BC_PERIODIC", "dirichlet": "DGSRHD_BC_DIRICHLET",
               "outflow": "DGSRHD_BC_OUTFLOW", "reflect": "DGSRHD_BC_REFLECT"},
        "PRECISION": {"fp64": "DGSRHD_PREC_FP64", "split": "DGSRHD_PREC_SPLIT",
                      "3xtf32": "DGSRHD_PREC_3XTF32"},
        "NODES": {"gl": "DGSRHD_NODES_GL", "gll": "DGSRHD_NODES_GLL"},
        "LIMITER": {"none": "DGSRHD_LIMITER_NONE", "moe": "DGSRHD_LIMITER_SCALING",
                    "scaling": "DGSRHD_LIMITER_SCALING", "minmod": "DGSRHD_LIMITER_MINMOD"},
        "ENFORCE": {"off": "DGSRHD_ENFORCE_OFF", "nodes": "DGSRHD_ENFORCE_NODES",
                    "faces": "DGSRHD_ENFORCE_FACES"},
        "PROBE": {"dfma": "DGSRHD_PROBE_DFMA", "ddiv": "DGSRHD_PROBE_DDIV",
                  "dsqrt": "DGSRHD_PROBE_DSQRT", "drsqrt": "DGSRHD_PROBE_DRSQRT",
                  "drcbrt": "DGSRHD_PROBE_DRCBRT", "recip": "DGSRHD_PROBE_RECIP",
                  "sqrt": "DGSRHD_PROBE_SQRT", "rcbrt": "DGSRHD_PROBE_RCBRT",
                  "ffma": "DGSRHD_PROBE_FFMA", "rsqrt": "DGSRHD_PROBE_RSQRT"},
    }
    for group, names in groups.items():
        table = getattr(_lib, group)
        assert set(table) == set(names), group
        for key, const in names.items():
            assert table[key] == c[const], (group, key)


def header_prototypes():
    """{name: (return type, [parameter types])} of every function include/dgsrhd.h declares."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = {}
    for ret, name, params in re.findall(
            r"^\s*((?:const\s+)?[a-z_0-9]+\s*\**)\s*(dgsrhd_[a-z_0-9]+)\s*\(([^)]*)\)\s*;",
            text, flags=re.M):
        types = []
        for prm in params.split(","):
            prm = " ".join(prm.split())
            if prm in ("", "void"):
                continue
            # drop the parameter's name: the last identifier not followed by '*'
            types.append(re.sub(r"\s*\b[a-zA-Z_][a-zA-Z_0-9]*$", "", prm).replace(" *", "*"))
        protos[name] = (" ".join(ret.split()).replace(" *", "*"), types)
    return protos


SCALARS = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double}
POINTEES = dict(SCALARS, dgsrhd_config=_lib.dgsrhd_config, dgsrhd_stats=_lib.dgsrhd_stats)


def _check_type(ctype, ctext, where):
    ctext = ctext.replace("const ", "")
    if ctext.endswith("*"):
        pointee = ctext[:-1].strip()
        if ctype is ctypes.c_void_p:
            return  # an address: any pointer
        if ctype is ctypes.c_char_p:
            assert pointee == "char", where
            return
        assert hasattr(ctype, "_type_") and issubclass(ctype, ctypes._Pointer), where
        if pointee.endswith("*"):     # a pointer to a pointer (an out-handle)
            assert ctype._type_ is ctypes.c_void_p, where
        else:
            assert ctype._type_ is POINTEES[pointee], where
    elif ctext == "void":
        assert ctype is None, where
    else:
        assert ctype is SCALARS[ctext], where


def test_function_signatures_match_the_header():
    lib = _lib.load()
    protos = header_prototypes()
    assert sorted(protos) == sorted(_lib.exported_symbols())
    for name, (ret, params) in protos.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None and len(fn.argtypes) == len(params), name
        _check_type(fn.restype, ret, f"{name} return")
        for k, (ct, pt) in enumerate(zip(fn.argtypes, params)):
            _check_type(ct, pt, f"{name} argument {k}")
