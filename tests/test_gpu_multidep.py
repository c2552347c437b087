"""GPU parity of the commutative-multidependence assembly (Sec. 3.2.2, Alg.
"multideps"): subdomains of `chunk` elements run under locks on their whole
neighbour lists, elements in local color classes, plain read-modify-write.
Checks the result against the oracle, the plan against brute force, that no
two subdomains whose lists meet ever ran at the same time, and the bounded
wait when a lock is never released."""
import numpy as np
import pytest

from paper_1805_03949_gb300 import meshgen as mg
from tests.helpers import FP32_TOL, FP64_TOL, engine, err_vs_oracle

pytestmark = pytest.mark.gpu

_REF = {}
_MESHES = {
    "hex9": lambda: mg.hex_cube(9, 0.2, 2),
    "hybrid4": lambda: mg.hybrid_cube(4, 5),
    "kuhn5": lambda: mg.kuhn_tet_cube(5),
    "ragged": lambda: mg.hex_cube(0, 0.2, 5, nx=3, ny=1, nz=7),
}


def _ref(oracle, name, mesh, kind):
    key = (name, kind)
    if key not in _REF:
        _REF[key] = oracle.assemble(mesh, kind, tet_rule=1, poisson=0.3, k0=1.0, k2=1.0)
    return _REF[key]


def _assemble(fea, s, kind, precision, chunk, **kw):
    op = fea.make_operator(kind=kind, precision=precision, scatter=fea.FEA_SCATTER_MULTIDEP, tet_rule=1,
                           poisson=0.3, k0=1.0, k2=1.0, chunk=chunk, **kw)
    s.A.fill_(float("nan"))
    s.b.fill_(float("nan"))
    s.assemble(op)
    return op


@pytest.mark.parametrize("name", list(_MESHES))
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("chunk", [1, 7, 128])
def test_multidep_matches_oracle(oracle, name, kind, precision, chunk):
    fea = engine()
    mesh = _MESHES[name]()
    s = fea.System.from_mesh(mesh, 1 if kind == 0 else 3)
    try:
        _assemble(fea, s, kind, precision, chunk)
        s.check()
        ref = _ref(oracle, name, mesh, kind)
        tol = FP64_TOL if precision == 0 else FP32_TOL
        errA, zA = err_vs_oracle(s.A.cpu().numpy(), ref["A"], ref["NA"])
        errb, zb = err_vs_oracle(s.b.cpu().numpy(), ref["b"], ref["Nb"])
        assert max(errA, errb, zA, zb) <= tol, (errA, errb, zA, zb)
    finally:
        s.close()


def _subdomains(mesh, chunk):
    """Work items of `chunk` elements per type (enum order, upload order):
    the element ids of each subdomain, independent of the engine."""
    subs = []
    for t in range(4):
        ids = np.nonzero(mesh.types == t)[0]
        for f in range(0, len(ids), chunk):
            subs.append(ids[f:f + chunk])
    return subs


@pytest.mark.parametrize("name,chunk", [("hybrid4", 7), ("hex9", 16), ("kuhn5", 1)])
def test_plan_matches_brute_force(name, chunk):
    fea = engine()
    mesh = _MESHES[name]()
    s = fea.System.from_mesh(mesh, 1)
    try:
        plan = fea.fea_multidep_plan(s.handle, chunk, mesh.n_elems)
        subs = _subdomains(mesh, chunk)
        assert plan["subdomains"] == len(subs)
        off = mesh.conn_offsets
        nodes = [set(np.concatenate([mesh.conn[off[e]:off[e + 1]] for e in sub]).tolist()) for sub in subs]
        for k in range(len(subs)):
            want = [j for j in range(len(subs)) if nodes[k] & nodes[j]]
            got = plan["nb"][plan["nb_off"][k]:plan["nb_off"][k + 1]].tolist()
            assert got == want, k
        deg = np.diff(plan["nb_off"])
        order = plan["order"]
        assert sorted(order.tolist()) == list(range(len(subs)))
        assert (np.diff(deg[order]) <= 0).all()          # more neighbours first
        # local colors: inside a subdomain, elements of one color share no node
        col = plan["color"]
        for sub in subs:
            for c in np.unique(col[sub]):
                members = sub[col[sub] == c]
                allnodes = np.concatenate([mesh.conn[off[e]:off[e + 1]] for e in members])
                assert len(allnodes) == len(np.unique(allnodes))
        assert col.min() >= 0 and plan["max_colors"] == col.max() + 1
    finally:
        s.close()


@pytest.mark.parametrize("chunk", [1, 8, 64])
def test_conflicting_subdomains_never_overlap(chunk):
    """Per lock, the subdomains that take it ran one after the other (their
    take-to-last-add %globaltimer spans are disjoint)."""
    import torch
    fea = engine()
    mesh = mg.hex_cube(12, 0.2, 3)
    s = fea.System.from_mesh(mesh, 3)
    try:
        plan = fea.fea_multidep_plan(s.handle, chunk, mesh.n_elems)
        n = plan["subdomains"]
        span = torch.zeros(2 * n, dtype=torch.int64, device="cuda")
        _assemble(fea, s, 1, 1, chunk, span=span)
        s.check()
        sp = span.cpu().numpy().reshape(n, 2)
        assert (sp[:, 0] > 0).all() and (sp[:, 1] >= sp[:, 0]).all()
        nb_off, nb = plan["nb_off"], plan["nb"]
        users = {}
        for k in range(n):
            for j in nb[nb_off[k]:nb_off[k + 1]]:
                users.setdefault(int(j), []).append(k)
        overlaps = 0
        for lock, ks in users.items():
            iv = sp[ks]
            iv = iv[np.argsort(iv[:, 0], kind="stable")]
            overlaps += int((iv[1:, 0] < iv[:-1, 1]).sum())
        assert overlaps == 0
        # many subdomains did run at the same time (the locks are not a global one)
        ev = np.concatenate([np.stack([sp[:, 0], np.ones(n)], 1), np.stack([sp[:, 1], -np.ones(n)], 1)])
        ev = ev[np.lexsort((ev[:, 1], ev[:, 0]))]
        assert np.cumsum(ev[:, 1]).max() > 1
    finally:
        s.close()


def test_held_lock_times_out_and_the_context_stays_usable(oracle):
    fea = engine()
    mesh = mg.hex_cube(6, 0.2, 4)
    s = fea.System.from_mesh(mesh, 3)
    try:
        fea.fea_multidep_plan(s.handle, 8, mesh.n_elems)
        fea.fea_multidep_hold(s.handle, 3, True)
        _assemble(fea, s, 1, 1, 8, lock_timeout_us=20000)
        with pytest.raises(fea.FeaError) as e:
            s.check()
        assert e.value.code == -6  # FEA_ERR_TIMEOUT
        fea.fea_multidep_hold(s.handle, 3, False)
        _assemble(fea, s, 1, 1, 8, lock_timeout_us=20000)
        s.check()
        ref = _ref(oracle, "hex6", mesh, 1)
        errA, zA = err_vs_oracle(s.A.cpu().numpy(), ref["A"], ref["NA"])
        assert max(errA, zA) <= FP32_TOL
    finally:
        s.close()
