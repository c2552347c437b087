"""The C-ABI library loads and exports every function the header declares (no GPU).

Only calls that fail argument validation before touching the device are made.
"""
import ctypes
import os
import re

import pytest

from paper_1805_03949_gb300 import build
from tests.helpers import engine

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


def test_every_entry_point_rejects_a_null_handle(clib):
    """Each call with a null handle (or null required output) fails with
    FEA_ERR_ARG before touching the device; so do out-of-range sizes."""
    I64, F = ctypes.c_int64, ctypes.c_float
    n = ctypes.c_int64()
    k = ctypes.c_int()
    info = (ctypes.c_int64 * 8)()
    out = ctypes.c_void_p()
    calls = {
        "fea_mesh_set_coords": (None, None, 0, None),
        "fea_mesh_destroy": (None,),
        "fea_pattern_size": (None, 3, ctypes.byref(n), None),
        "fea_build_csr_pattern": (None, 3, None, None, None, None),
        "fea_work_items": (None, 0, ctypes.byref(n), None, None, None),
        "fea_persistent_grid": (None, None, ctypes.byref(k)),
        "fea_element_loop": (None, None, None, None),
        "fea_element_loop_grid": (None, None, ctypes.byref(k)),
        "fea_costmodel_destroy": (None,),
        "fea_costmodel_get_params": (None, None, None),
        "fea_costmodel_fit_scaler": (None, None, None, I64(0), None),
        "fea_costmodel_grad": (None, None, None, I64(1), None, None, None),
        "fea_costmodel_train": (None, None, None, I64(1), 1, F(0.01), None, None),
        "fea_costmodel_predict": (None, None, I64(0), None, None),
        "fea_item_features": (None, 0, None, None, None, None),
        "fea_batch_create": (None, 1, None, ctypes.byref(out)),
        "fea_batch_destroy": (None,),
        "fea_batch_set_config": (None, 64, 0),
        "fea_batch_info": (None, None, None, None),
        "fea_batch_autotune": (None, 1, None, None, None, None),
        "fea_batch_capture": (None, None),
        "fea_batch_assemble": (None, None),
        "fea_batch_latency": (None, None, None),
        "fea_row_ptr_from_counts_noalloc": (None, I64(-1), None, None),
        "fea_mesh_set_rows_block": (None, 64),
        "fea_mesh_set_block_elems": (None, 64),
        "fea_rows_plan_info": (None, info),
        "fea_color_info": (None, None, ctypes.byref(k)),
        "fea_assemble_launches": (None, None, ctypes.byref(k)),
        "fea_pack_lpt": (None, I64(1), 1, None, None, None),
        "fea_peak_probe": (0, I64(1000), None, None),
        "fea_convert": (2, None, None, I64(0), None),
        "fea_mesh_set_pipe_split": (None, 6),
        "fea_autotune": (None, None, None, None, None, None, 3, None, None),
    }
    for name, args in calls.items():
        assert getattr(clib, name)(*args) == -1, name
    params = (ctypes.c_float * 2048)()
    for n_in in (0, 9):                                   # the network takes 1..8 features
        assert clib.fea_costmodel_create(n_in, params, ctypes.byref(out)) == -1
    assert not out.value


def test_binding_structs_match_the_header(tmp_path):
    """sizeof and field offsets of the ctypes structs equal the C compiler's view of the header."""
    from paper_1805_03949_gb300 import fea
    probe = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fea_gb300.h"', 'int main(void) {']
    structs = {"fea_operator": fea.fea_operator, "fea_mesh_desc": fea.fea_mesh_desc,
               "fea_batch_entry": fea.fea_batch_entry, "fea_tuning": fea.fea_tuning}
    for cname, cls in structs.items():
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
        cls = structs[cname]
        expect = ctypes.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert int(value) == expect, (cname, field, value, expect)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())


@pytest.mark.gpu
def test_binding_checks_pointer_types_and_sizes():
    """The binding refuses a tensor whose dtype or length the C side would misread or overrun."""
    fea = engine()
    import torch
    counts = torch.ones(10, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        fea.fea_row_ptr_from_counts_noalloc(counts, torch.zeros(10, dtype=torch.int64, device="cuda"))
    with pytest.raises(TypeError):
        fea.fea_row_ptr_from_counts_noalloc(counts.to(torch.int64), torch.zeros(11, dtype=torch.int64,
                                                                                device="cuda"))
    with pytest.raises(TypeError):
        fea.fea_row_ptr_from_counts_noalloc(counts, torch.zeros(11, dtype=torch.int32, device="cuda"))
    with pytest.raises(TypeError):
        fea.fea_row_ptr_from_counts_noalloc(counts.cpu(), torch.zeros(11, dtype=torch.int64))


def test_peak_probe_rejects_bad_arguments(clib):
    f = ctypes.c_double()
    assert clib.fea_peak_probe(2, ctypes.c_int64(1000), ctypes.byref(f), None) == -1
    assert clib.fea_peak_probe(0, ctypes.c_int64(3), ctypes.byref(f), None) == -1


@pytest.mark.gpu
def test_peak_probe_measures_the_fma_rates():
    """FP64 near GB300's nominal 1.25 TFLOP/s (2 FP64 FMA per SM and clock),
    FP32 near 152 SMs x 128 lanes x 2 flop x clock; FP32 far above FP64."""
    fea = engine()
    p64 = fea.fea_peak_probe(0, 20000)
    p32 = fea.fea_peak_probe(1, 200000)
    assert 0.6e12 < p64 < 1.5e12, p64
    assert 40e12 < p32 < 90e12, p32
    assert p32 > 30 * p64
