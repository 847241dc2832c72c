"""The C-ABI library loads and exports every symbol that include/nebem.h declares.

CPU-only: no compute call is made (there is no GPU here); creating a context must fail
with NEBEM_NO_DEVICE rather than fall back to anything.
"""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nebem.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nebem_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_24154_gb300 import build, nebem
    build.build()
    return nebem.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2606_24154_gb300 import nebem
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
        assert name in nebem.SIGNATURES, f"binding lacks {name}"
    out = subprocess.run(["nm", "-D", "--defined-only", nebem.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (nebem_\w+)", out))
    assert set(names) <= exported, set(names) - exported


def test_no_device_is_an_error_not_a_fallback(lib):
    import torch
    from paper_2606_24154_gb300 import nebem
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(nebem.NebemError) as ei:
        nebem.nebem_create()
    assert ei.value.code == nebem.NEBEM_NO_DEVICE


def test_status_strings_and_defaults(lib):
    from paper_2606_24154_gb300 import nebem
    assert lib.nebem_status_string(nebem.NEBEM_SINGULAR) == b"NEBEM_SINGULAR"
    o = nebem.nebem_default_options()
    assert o.ir_tol == 1e-8 and o.lu_block == 64 and o.softening == 1e-6
    assert o.mixed_point_tol == 1e-6


@pytest.mark.parametrize("field,value", [
    ("lu_block", 48), ("lu_block", 16), ("lu_block", 128),
    ("ir_max_iter", 0), ("ir_tol", 0.0), ("ir_tol", float("nan")),
    ("ratio_near", 1.0), ("ratio_b", 2.0), ("ratio_a", 7.0), ("ratio_0", 20.0), ("ratio_0", 1e7),
    ("softening", 0.0), ("softening", -1e-6),
    ("mixed_point_tol", -1e-6), ("mixed_point_tol", 1.0), ("mixed_point_tol", float("nan")),
    ("wait_polls", -1),
])
def test_bad_options_refused_before_any_device_call(lib, field, value):
    """Context options are checked on the host before the device is touched: every bad
    value is NEBEM_INVALID_ARG (with or without a GPU), never a silently corrected
    default.  The tier ratios must keep 1.5 <= ratio_near <= ratio_b <= ratio_a <= ratio_0."""
    from paper_2606_24154_gb300 import nebem
    o = nebem.nebem_default_options()
    setattr(o, field, value)
    with pytest.raises(nebem.NebemError) as ei:
        nebem.nebem_create(o)
    assert ei.value.code == nebem.NEBEM_INVALID_ARG
    assert lib.nebem_last_error() != b""


def test_oracle_and_product_share_no_code():
    """The oracle and the CUDA path are independent: no Python module of the package
    imports oracle/, the oracle imports nothing of the package, and neither side's C/CUDA
    sources include the other's headers.  Only the seeded input generators are shared
    (by the tests and the bench, not by either implementation)."""
    import ast
    pkg = os.path.join(ROOT, "paper_2606_24154_gb300")
    orc = os.path.join(ROOT, "oracle")

    def py_imports(path):
        names = set()
        for node in ast.walk(ast.parse(open(path).read())):
            if isinstance(node, ast.Import):
                names |= {a.name for a in node.names}
            elif isinstance(node, ast.ImportFrom):
                names.add(("." * node.level) + (node.module or ""))
        return names

    for f in os.listdir(pkg):
        if f.endswith(".py"):
            assert not any(n.split(".")[0].lstrip(".") == "oracle" for n in py_imports(os.path.join(pkg, f))), f
    for f in os.listdir(orc):
        if f.endswith(".py"):
            assert not any("paper_2606_24154_gb300" in n for n in py_imports(os.path.join(orc, f))), f
    csrc = os.path.join(pkg, "csrc")
    for f in os.listdir(csrc):
        inc = re.findall(r'#include\s+"([^"]+)"', open(os.path.join(csrc, f)).read())
        assert all("oracle" not in i for i in inc), (f, inc)
    for f in os.listdir(orc):
        if f.endswith((".c", ".h")):
            inc = re.findall(r'#include\s+[<"]([^">]+)[">]', open(os.path.join(orc, f)).read())
            assert all(i in {"math.h", "stdint.h", "stdlib.h", "string.h", "omp.h", "stdio.h"} for i in inc), (f, inc)


def test_missing_library_fails_loudly():
    """Without libnebem.so the binding raises: no call falls back to another code path."""
    import subprocess
    import sys
    code = ("from paper_2606_24154_gb300 import nebem\n"
            "try:\n"
            "    nebem.load('/nonexistent/libnebem.so')\n"
            "except RuntimeError as e:\n"
            "    print('raised', 'not found' in str(e))\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.stdout.strip() == "raised True", r.stdout + r.stderr
