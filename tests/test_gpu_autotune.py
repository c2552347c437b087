"""The autotuner and the producer/consumer split of the pipelined block-task
kernel: every configuration the autotuner may choose assembles the same
system as the oracle, and the choice comes from the documented candidates."""
import json

import numpy as np
import pytest

from paper_1805_03949_gb300 import meshgen as mg
from tests.helpers import FP32_TOL, engine, err_vs_oracle

pytestmark = pytest.mark.gpu

_REF = {}


def _ref(oracle, name, mesh, op, **kw):
    if name not in _REF:
        _REF[name] = oracle.assemble(mesh, op, **kw)
    return _REF[name]


def _check(s, ref):
    errA, zA = err_vs_oracle(s.A.cpu().numpy(), ref["A"], ref["NA"])
    errb, zb = err_vs_oracle(s.b.cpu().numpy(), ref["b"], ref["Nb"])
    assert max(errA, zA, errb, zb) <= FP32_TOL, (errA, zA, errb, zb)


@pytest.mark.parametrize("name", ["hex9", "ragged_hex"])
@pytest.mark.parametrize("block_elems", [32, 64, 80])
def test_every_pipe_split_matches_oracle(oracle, name, block_elems):
    """Producer warps 4..8 (4 x warps elements per geometry pass, ragged last
    passes), blocks of 32..80 elements, against the FP64 oracle."""
    fea = engine()
    mesh = mg.hex_cube(9, 0.2, 2) if name == "hex9" else mg.hex_cube(0, 0.2, 5, nx=7, ny=5, nz=3)
    ref = _ref(oracle, name, mesh, oracle.OP_ELASTICITY, young=1.0, poisson=0.3)
    s = fea.System.from_mesh(mesh, 3)
    try:
        fea.fea_mesh_set_block_elems(s.handle, block_elems)
        op = fea.make_operator(kind=1, precision=1, scatter=fea.FEA_SCATTER_BLOCK, poisson=0.3)
        for pw in range(4, 9):
            fea.fea_mesh_set_pipe_split(s.handle, pw)
            s.A.fill_(float("nan"))
            s.assemble(op)
            s.check()
            _check(s, ref)
    finally:
        s.close()


def test_pipe_split_range_is_checked():
    fea = engine()
    s = fea.System.from_mesh(mg.hex_cube(2, 0.0), 3)
    try:
        for bad in (3, 9):
            with pytest.raises(fea.FeaError):
                fea.fea_mesh_set_pipe_split(s.handle, bad)
    finally:
        s.close()


CASES = {
    # name: (mesh, op kwargs, oracle op, oracle kwargs, the tuned field and its candidates)
    "block_hex": (lambda: mg.hex_cube(10, 0.2, 2), dict(kind=1, precision=1, scatter=2, poisson=0.3), 1,
                  dict(young=1.0, poisson=0.3), ("block_elems", {32, 48, 64, 80})),
    "rows_hybrid": (lambda: mg.hybrid_cube(6, 3), dict(kind=0, precision=1, scatter=3, k0=1.0, k2=1.0, source=1.0),
                    0, dict(k0=1.0, k2=1.0, source=1.0), ("rows_block_nodes", {32, 64, 96, 128})),
    "steal_hybrid": (lambda: mg.hybrid_cube(6, 3), dict(kind=1, precision=1, schedule=1, poisson=0.3), 1,
                     dict(young=1.0, poisson=0.3), ("chunk", {16, 32, 64, 128, 256})),
    "multidep_hex": (lambda: mg.hex_cube(10, 0.2, 2), dict(kind=1, precision=1, scatter=4, poisson=0.3), 1,
                     dict(young=1.0, poisson=0.3), ("chunk", {64, 128, 256})),
}


@pytest.mark.parametrize("name", list(CASES))
def test_autotuned_configuration_matches_oracle(oracle, name, tmp_path):
    fea = engine()
    factory, kw, oop, okw, (field, cands) = CASES[name]
    mesh = factory()
    ref = _ref(oracle, name, mesh, oop, **okw)
    s = fea.System.from_mesh(mesh, 1 if kw["kind"] == 0 else 3)
    try:
        op = fea.make_operator(**kw)
        cache = str(tmp_path / "tuning.json")
        t = fea.autotune(op, s, key=name, cache=cache, reps=2)
        assert not t["cached"] and t[field] in cands and t["ms"] > 0
        if name == "block_hex":
            assert t["producer_warps"] in range(4, 9) and t["candidates"] == 20
        _check(s, ref)                                   # the autotuner leaves an assembly with its choice
        s.A.fill_(float("nan"))
        s.assemble(op)
        s.check()
        _check(s, ref)
        # the cache applies the same choice without timing
        op2 = fea.make_operator(**kw)
        t2 = fea.autotune(op2, s, key=name, cache=cache)
        assert t2["cached"] and t2[field] == t[field] and op2.chunk == op.chunk
        assert json.load(open(cache))[name][field] == t[field]
    finally:
        s.close()


def test_assemble_refuses_misaligned_values():
    """A must be 16-byte aligned (rows of complete entry blocks are written
    with 16-byte stores); an offset view is refused before any work."""
    import torch
    fea = engine()
    s = fea.System.from_mesh(mg.hex_cube(2, 0.0), 3)
    try:
        op = fea.make_operator(kind=1, precision=1, scatter=fea.FEA_SCATTER_BLOCK, poisson=0.3)
        buf = torch.zeros(s.A.numel() + 1, dtype=torch.float64, device="cuda")
        with pytest.raises(fea.FeaError):
            fea.fea_assemble(op, s.handle, s.row_ptr, s.node_map, buf[1:], s.b)
        s.assemble(op)
        s.check()
    finally:
        s.close()
