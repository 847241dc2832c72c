"""The Python binding matches the C-ABI exactly, CPU only: every function's argument
count and scalar widths in nebem.py's ctypes table agree with include/nebem.h (a typed
pointer in the binding points to the declared type), and every struct the calls take has
the same size and field offsets in C (compiled here with gcc) as in the binding's ctypes
structures and the element record dtype."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2606_24154_gb300 import inputs as I
from paper_2606_24154_gb300 import nebem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nebem.h")

SCALARS = {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double, "int": C.c_int}
POINTEES = {"double": C.c_double, "float": C.c_float, "int64_t": C.c_int64, "int32_t": C.c_int32,
            "uint8_t": C.c_uint8, "nebem_options": nebem.nebem_options,
            "nebem_solve_info": nebem.nebem_solve_info, "nebem_server_options": nebem.nebem_server_options}


def declarations():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\b(int|const char \*)\s*(nebem_\w+)\s*\(([^;]*?)\)\s*;", src, re.S):
        ret, name, params = m.group(1), m.group(2), " ".join(m.group(3).split())
        out[name] = (ret, [] if params in ("", "void") else [p.strip() for p in params.split(",")])
    return out


def _check_param(name, i, decl, ctype):
    stars = decl.count("*")
    base = re.sub(r"\b(const|restrict)\b", "", decl.split("*")[0]).split()
    base = base[0] if base else ""
    if stars == 0:
        assert ctype is SCALARS[base], (name, i, decl, ctype)
        return
    # any pointer: c_void_p, or a typed pointer to the declared type
    if ctype is C.c_void_p:
        return
    assert issubclass(ctype, C._Pointer), (name, i, decl, ctype)
    pointee = ctype._type_
    if stars == 2:
        assert pointee is C.c_void_p, (name, i, decl, ctype)
    elif base in POINTEES:
        assert pointee is POINTEES[base], (name, i, decl, ctype)


def test_signatures_match_the_header():
    decl = declarations()
    assert set(decl) == set(nebem.SIGNATURES), set(decl) ^ set(nebem.SIGNATURES)
    for name, (ret, params) in decl.items():
        res, args = nebem.SIGNATURES[name]
        assert res is (C.c_int if ret == "int" else C.c_char_p), name
        assert len(args) == len(params), (name, params, args)
        for i, (p, a) in enumerate(zip(params, args)):
            _check_param(name, i, p, a)


STRUCTS = {
    "nebem_options": nebem.nebem_options,
    "nebem_solve_info": nebem.nebem_solve_info,
    "nebem_server_options": nebem.nebem_server_options,
}


def test_struct_layouts_match_c(tmp_path):
    gcc = "gcc"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nebem.h"', "int main(void) {"]
    for sname, cls in STRUCTS.items():
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines.append('printf("nebem_element size %zu\\n", sizeof(nebem_element));')
    for fname in I.ELEMENT_DTYPE.names:
        lines.append(f'printf("nebem_element {fname} %zu\\n", offsetof(nebem_element, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    try:
        subprocess.run([gcc, "-std=c11", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       check=True, capture_output=True, text=True)
    except FileNotFoundError:
        pytest.skip("no C compiler")
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for sname, cls in STRUCTS.items():
        assert got[(sname, "size")] == C.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[(sname, fname)] == getattr(cls, fname).offset, (sname, fname)
    assert got[("nebem_element", "size")] == I.ELEMENT_DTYPE.itemsize
    for fname in I.ELEMENT_DTYPE.names:
        assert got[("nebem_element", fname)] == I.ELEMENT_DTYPE.fields[fname][1], fname


def test_oracle_argtypes_match_its_c_definitions():
    """The same check for the oracle's own ctypes table (test infrastructure): argument
    count, scalar widths and pointee types of every exported function it declares."""
    from oracle import oracle as O
    src = open(os.path.join(ROOT, "oracle", "nebem_oracle.c")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    defs = {}
    for m in re.finditer(r"^(int|void|int64_t|double)\s+(or_\w+)\(([^)]*)\)\s*\{", src, re.M | re.S):
        params = " ".join(m.group(3).split())
        defs[m.group(2)] = (m.group(1), [] if params in ("", "void") else [p.strip() for p in params.split(",")])
    L = O.lib()
    checked = 0
    for name, (ret, params) in defs.items():
        f = getattr(L, name, None)
        if f is None or f.argtypes is None:
            continue
        assert len(f.argtypes) == len(params), (name, params, f.argtypes)
        for i, (p, a) in enumerate(zip(params, f.argtypes)):
            decl = re.sub(r"\b\w+\s*(\[\d*\])?$", lambda mm: "*" if mm.group(1) else "", p).strip()
            _check_param(name, i, decl if decl else p, a)
        if ret == "int64_t":
            assert f.restype is C.c_int64, name
        checked += 1
    assert checked >= 19, checked  # every function the oracle gives argtypes
