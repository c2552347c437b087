"""GPU parity of batched assembly: many meshes in one persistent launch, direct
and replayed as a CUDA graph, after autotuning; per-mesh latencies."""
import pytest

from paper_1805_03949_gb300 import meshgen as mg
from tests.helpers import FP32_TOL, FP64_TOL, engine, err_vs_oracle

pytestmark = pytest.mark.gpu

_REF = {}


def _meshes():
    ms = mg.batch_meshes(count=7, seed=5, lo=30, hi=3000)
    ms.append(mg.hybrid_cube(3, 5))                   # every element type in one entry
    return ms


def _check(oracle, key, mesh, s, tol, kind=1):
    if key not in _REF:
        _REF[key] = oracle.assemble(mesh, kind, tet_rule=1, poisson=0.3)
    ref = _REF[key]
    errA, zA = err_vs_oracle(s.A.cpu().numpy(), ref["A"], ref["NA"])
    errb, zb = err_vs_oracle(s.b.cpu().numpy(), ref["b"], ref["Nb"])
    assert errA <= tol and errb <= tol and zA <= tol and zb <= tol, (key, errA, errb, zA, zb)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_direct_graph_and_autotuned(oracle, precision):
    import torch
    fea = engine()
    meshes = _meshes()
    systems = [fea.System.from_mesh(m, 3) for m in meshes]
    tol = FP64_TOL if precision == 0 else FP32_TOL
    batch = None
    try:
        op = fea.make_operator(kind=1, precision=precision, tet_rule=1, poisson=0.3, chunk=16)
        batch = fea.Batch(op, systems)
        info = batch.info()
        assert info["items"] == sum(-(-int((m.types == t).sum()) // 16) for m in meshes for t in range(4))
        for s in systems:
            s.A.fill_(float("nan")); s.b.fill_(float("nan"))
        batch.assemble()
        torch.cuda.synchronize()
        for k, (m, s) in enumerate(zip(meshes, systems)):
            _check(oracle, k, m, s, tol)
        lat = batch.latency_ns()
        assert (lat > 0).all()
        # graph replay of the same assembly
        batch.capture()
        for s in systems:
            s.A.fill_(float("nan")); s.b.fill_(float("nan"))
        batch.assemble()
        batch.assemble()
        torch.cuda.synchronize()
        for k, (m, s) in enumerate(zip(meshes, systems)):
            _check(oracle, k, m, s, tol)
        # autotuned configuration, then a fresh graph
        best = batch.autotune(reps=1)
        assert best["chunk"] in (16, 32, 64, 128, 256, 512) and best["grid"] > 0 and best["ms"] > 0
        assert batch.info()["chunk"] == best["chunk"] and batch.info()["grid"] == best["grid"]
        batch.capture()
        for s in systems:
            s.A.fill_(float("nan"))
        batch.assemble()
        torch.cuda.synchronize()
        for k, (m, s) in enumerate(zip(meshes, systems)):
            _check(oracle, k, m, s, tol)
        for s in systems:
            s.check()
    finally:
        if batch is not None:
            batch.close()
        for s in systems:
            s.close()


def test_batch_rejects_mismatched_pattern():
    fea = engine()
    s = fea.System.from_mesh(mg.hex_cube(2), 1)
    try:
        with pytest.raises(fea.FeaError):
            fea.Batch(fea.make_operator(kind=1), [s])
    finally:
        s.close()
