"""The C-ABI library loads and exports every function the header declares (no GPU).

Only calls that fail argument validation before touching the device are made.
"""
import ctypes
import os
import re

import pytest

from paper_1805_03949_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(fea_[a-z0-9_]+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def clib():
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["fea_mesh_upload", "fea_build_csr_pattern", "fea_assemble", "fea_pattern_size",
                     "fea_check", "fea_last_error", "fea_mesh_destroy", "fea_mesh_info"]:
        assert required in names


def test_every_declared_symbol_is_exported(clib):
    for name in _declared():
        assert hasattr(clib, name), name


def test_host_side_argument_checks(clib):
    clib.fea_abi_version.restype = ctypes.c_int
    assert clib.fea_abi_version() == 3
    clib.fea_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    rc = clib.fea_mesh_upload(None, None, ctypes.byref(out))
    assert rc == -1                                   # FEA_ERR_ARG
    assert b"null" in clib.fea_last_error()
    n = ctypes.c_int64()
    assert clib.fea_mesh_info(None, ctypes.byref(n), None, None) == -1
    assert clib.fea_assemble(None, None, None, None, None, None, None) == -1
    assert clib.fea_check(None, None) == -1
    # the product, the multidependence plan and its test hook reject a null mesh
    assert clib.fea_spmv(None, 3, None, None, None, None, None, None, None) == -1
    info = (ctypes.c_int64 * 4)()
    assert clib.fea_multidep_plan(None, 0, info, None, None, None, None) == -1
    assert clib.fea_multidep_hold(None, 0, 1) == -1
    assert b"multidep" in clib.fea_last_error()


def test_binding_structs_match_the_header(tmp_path):
    """sizeof and field offsets of the ctypes structs equal the C compiler's view of the header."""
    from paper_1805_03949_gb300 import fea
    probe = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fea_gb300.h"', 'int main(void) {']
    for cname, cls in (("fea_operator", fea.fea_operator), ("fea_mesh_desc", fea.fea_mesh_desc)):
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines.append("return 0; }")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    seen = 0
    for line in out:
        if not line:
            continue
        cname, field, value = line.split()
        cls = fea.fea_operator if cname == "fea_operator" else fea.fea_mesh_desc
        expect = ctypes.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert int(value) == expect, (cname, field, value, expect)
        seen += 1
    assert seen == len(fea.fea_operator._fields_) + len(fea.fea_mesh_desc._fields_) + 2
