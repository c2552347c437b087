"""GPU parity of the persistent schedules (work stealing, static queues) and of
the elastoplastic J2 / Voce operator, through the C-ABI, against the CPU oracle.
"""
import numpy as np
import pytest

from paper_1805_03949_gb300 import meshgen as mg
from tests.helpers import FP32_TOL, FP64_TOL, engine, err_vs_oracle, j2_point_errors

pytestmark = pytest.mark.gpu

SCHED_CASES = {
    "kuhn8_poisson_tet1": (lambda: mg.kuhn_tet_cube(8), 0, 0, dict(k0=1.0, k2=0.0, source=1.0)),
    "hybrid6_diffusion": (lambda: mg.hybrid_cube(6, 3), 0, 1, dict(k0=1.0, k2=1.0, source=1.0)),
    "hybrid5_elasticity": (lambda: mg.hybrid_cube(5, 4), 1, 1, dict(young=2.0, poisson=0.25)),
    "ragged_hex_elasticity": (lambda: mg.hex_cube(0, 0.2, 5, nx=3, ny=4, nz=5), 1, 1, dict(poisson=0.3)),
}
_REF = {}


def _queues(n_items, n_ctas, seed):
    """A random assignment of every item to one of n_ctas queues (offsets, ids)."""
    import torch
    rng = np.random.default_rng(seed)
    owner = rng.integers(0, n_ctas, n_items)
    order = np.argsort(owner, kind="stable")
    off = np.zeros(n_ctas + 1, dtype=np.int64)
    np.add.at(off, owner + 1, 1)
    off = np.cumsum(off)
    return (torch.tensor(order.astype(np.int32), device="cuda"), torch.tensor(off, device="cuda"))


@pytest.mark.parametrize("chunk", [1, 7, 0])
@pytest.mark.parametrize("schedule", ["steal", "queues", "queues_steal"])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(SCHED_CASES))
def test_persistent_schedules_match_oracle(oracle, name, precision, schedule, chunk):
    import torch
    fea = engine()
    factory, kind, tet_rule, params = SCHED_CASES[name]
    mesh = factory()
    s = fea.System.from_mesh(mesh, 1 if kind == 0 else 3)
    try:
        _, _, counts = fea.fea_work_items(s.handle, chunk)
        n_items = len(counts)
        assert counts.sum() == mesh.n_elems
        item_ns = torch.zeros(n_items, dtype=torch.int64, device="cuda")
        item_cta = torch.full((n_items,), -1, dtype=torch.int32, device="cuda")
        kw = dict(kind=kind, precision=precision, tet_rule=tet_rule, chunk=chunk, item_ns=item_ns,
                  item_cta=item_cta, **params)
        if schedule == "steal":
            op = fea.make_operator(schedule=fea.FEA_SCHED_STEAL, **kw)
            grid = fea.fea_persistent_grid(op, s.handle)
        else:
            grid = 5
            q, qo = _queues(n_items, grid, 11)
            mode = fea.FEA_SCHED_QUEUES if schedule == "queues" else fea.FEA_SCHED_QUEUES_STEAL
            op = fea.make_operator(schedule=mode, n_ctas=grid, queue=q, queue_off=qo, **kw)
        s.A.fill_(float("nan"))
        s.assemble(op)
        s.check()
        assert fea.fea_assemble_launches(op, s.handle) == 1
        if name not in _REF:
            _REF[name] = oracle.assemble(mesh, 0 if kind == 0 else 1, tet_rule=tet_rule, **params)
        ref = _REF[name]
        tol = FP64_TOL if precision == 0 else FP32_TOL
        errA, zA = err_vs_oracle(s.A.cpu().numpy(), ref["A"], ref["NA"])
        errb, zb = err_vs_oracle(s.b.cpu().numpy(), ref["b"], ref["Nb"])
        assert errA <= tol and errb <= tol and zA <= tol and zb <= tol, (errA, errb, zA, zb)
        # every item ran once, on a CTA of the grid, and recorded a duration
        cta = item_cta.cpu().numpy()
        assert (cta >= 0).all() and (cta < grid).all()
        assert (item_ns.cpu().numpy() > 0).all()
        if schedule == "queues":
            qn = q.cpu().numpy(); qoff = qo.cpu().numpy()
            for c in range(grid):
                assert (cta[qn[qoff[c]:qoff[c + 1]]] == c).all()
    finally:
        s.close()


# ---------------------------------------------------------------------------
# J2 / Voce
# ---------------------------------------------------------------------------

J2_CASES = {
    # amplitudes chosen (with the oracle) for a mixed elastic / plastic second step
    "hex5": (lambda: mg.hex_cube(5, 0.2, 4), 1.5e-4),
    "hex1x2x9_ragged": (lambda: mg.hex_cube(0, 0.2, 8, nx=1, ny=2, nz=9), 1e-4),
    "tet3": (lambda: mg.template_cube(3, mg.TET4, 0.2, 8), 1.5e-4),
    "prism3": (lambda: mg.template_cube(3, mg.PRISM6, 0.2, 8), 1.5e-4),
    "pyr2": (lambda: mg.template_cube(2, mg.PYR5, 0.2, 8), 1.5e-4),
    "hybrid3": (lambda: mg.hybrid_cube(3, 5), 1.5e-4),
}
_J2REF = {}


def _j2_gpu(fea, s, U, precision, scatter=0, schedule=0, state_in=None):
    import torch
    E = s.n_elems
    u = torch.tensor(U.reshape(-1), device="cuda")
    st_out = torch.full((E, 8, 7), float("nan"), dtype=torch.float64, device="cuda")
    yl = torch.full((E, 8), 255, dtype=torch.uint8, device="cuda")
    it = torch.full((E, 8), 255, dtype=torch.uint8, device="cuda")
    op = fea.make_operator(kind=fea.FEA_OP_J2, precision=precision, scatter=scatter, schedule=schedule,
                           u=u, state_in=state_in, state_out=st_out, yield_out=yl, iters_out=it)
    s.A.fill_(float("nan"))
    s.assemble(op)
    s.check()
    return s.A.cpu().numpy(), s.b.cpu().numpy(), st_out, yl.cpu().numpy(), it.cpu().numpy()


def _nq(types):
    return np.array([4, 8, 6, 8])[types]


@pytest.mark.parametrize("variant", ["atomic", "color", "steal"])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(J2_CASES))
def test_j2_two_steps_match_oracle(oracle, name, precision, variant):
    fea = engine()
    factory, amp = J2_CASES[name]
    mesh = factory()
    U = mg.fourier_displacement(mesh.coords, amp, seed=4)
    if name not in _J2REF:
        r1 = oracle.j2_assemble(mesh, 0.5 * U)
        r2 = oracle.j2_assemble(mesh, U, r1["state"])
        p1 = oracle.j2_points(mesh, 0.5 * U)
        p2 = oracle.j2_points(mesh, U, r1["state"])   # the same update, with the stresses (per-point scales)
        _J2REF[name] = (r1, r2, p1, p2)
    r1, r2, p1, p2 = _J2REF[name]
    scatter = 1 if variant == "color" else 0
    schedule = 1 if variant == "steal" else 0
    s = fea.System.from_mesh(mesh, 3)
    try:
        _, _, st1, y1, _ = _j2_gpu(fea, s, 0.5 * U, precision, scatter, schedule)
        A, b, st2, y2, it2 = _j2_gpu(fea, s, U, precision, scatter, schedule, state_in=st1)
    finally:
        s.close()
    tol = FP64_TOL if precision == 0 else FP32_TOL
    errA, zA = err_vs_oracle(A, r2["A"], r2["NA"])
    errb, zb = err_vs_oracle(b, r2["b"], r2["Nb"])
    assert errA <= tol and errb <= tol and zA <= tol and zb <= tol, (errA, errb, zA, zb)
    mask = np.arange(8)[None, :] < _nq(mesh.types)[:, None]
    assert r2["yielded"][mask].any() and not r2["yielded"][mask].all()   # a mixed elastic / plastic state
    # the return map is FP64 in both precisions: every point's state (after
    # each step) at the FP64 bar of its own normwise scale, with no exemption
    assert np.array_equal(p1["state"], r1["state"]) and np.array_equal(p2["state"], r2["state"])
    err1, _ = j2_point_errors(st1.cpu().numpy(), None, r1["state"], p1["stress"], mask)
    err2, _ = j2_point_errors(st2.cpu().numpy(), None, r2["state"], p2["stress"], mask)
    y_mis = int((y1[mask] != r1["yielded"][mask]).sum()) + int((y2[mask] != r2["yielded"][mask]).sum())
    it_mis = int((it2[mask] != r2["iters"][mask]).sum())
    print(f"{name} precision {precision} {variant}: {int(mask.sum())} points, state err {err1:.2e} / {err2:.2e}, "
          f"yield mismatches {y_mis}, iteration mismatches {it_mis}")
    assert err1 <= FP64_TOL and err2 <= FP64_TOL, (err1, err2)
    assert y_mis <= 0.002 * mask.sum() and it_mis <= 0.01 * mask.sum(), (y_mis, it_mis)
    assert it2[mask].max() <= 12


def test_j2_no_convergence_is_reported(oracle):
    fea = engine()
    import torch
    mesh = mg.hex_cube(3, 0.2, 4)
    U = mg.fourier_displacement(mesh.coords, 1e-3, seed=4)
    s = fea.System.from_mesh(mesh, 3)
    try:
        u = torch.tensor(U.reshape(-1), device="cuda")
        op = fea.make_operator(kind=fea.FEA_OP_J2, u=u, max_iter=1, tol_step=0.0)
        s.assemble(op)
        with pytest.raises(fea.FeaError) as ei:
            s.check()
        assert ei.value.code == fea.FEA_ERR_NO_CONVERGENCE
        s.check()
    finally:
        s.close()
