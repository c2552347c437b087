"""GPU parity of the learned cost model (scaler, gradient, Adam, inference),
of the item features, and the makespan test of the MLP-packed persistent
schedule against Gauss-point-weight packing and work stealing.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_1805_03949_gb300 import meshgen as mg
from tests.helpers import engine

pytestmark = pytest.mark.gpu


def _data(n, seed=1):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 6))
    X[np.arange(n), rng.integers(0, 4, n)] = 1.0
    X[:, 4] = rng.uniform(0, 1, n)
    X[:, 5] = rng.lognormal(-8, 1, n)
    y = 3.0 + 0.5 * X[:, 0] + 1.5 * X[:, 4] + 1e3 * X[:, 5] + rng.normal(0, 0.05, n)
    return X.astype(np.float32), y.astype(np.float32)


def _tensors(X, y):
    import torch
    return torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda")


@pytest.mark.parametrize("n", [1, 255, 256, 1000, 4097])
def test_scaler_gradient_and_loss_match_oracle(n):
    fea = engine()
    X, y = _data(n)
    p0 = M.xavier_init(6).astype(np.float32)
    p0 = p0 + np.random.default_rng(2).normal(0, 0.05, p0.shape).astype(np.float32)
    h = fea.fea_costmodel_create(6, p0)
    try:
        Xd, yd = _tensors(X, y)
        fea.fea_costmodel_fit_scaler(h, Xd, yd)
        g, loss = fea.fea_costmodel_grad(h, Xd, yd, 1313)
        _, sc = fea.fea_costmodel_get_params(h, 6)
        xm, xs, ym, ys = M.fit_scaler(X.astype(np.float64), y.astype(np.float64))
        np.testing.assert_allclose(sc[:6], xm, rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(sc[6:12], xs, rtol=1e-5)
        np.testing.assert_allclose(sc[12:], [ym, ys], rtol=1e-5)
        # the oracle gradient at the same (FP32-rounded) scaler and parameters
        scd = (sc[:6].astype(np.float64), sc[6:12].astype(np.float64), float(sc[12]), float(sc[13]))
        lref, gref = M.loss_grad(p0.astype(np.float64), 6, X.astype(np.float64), y.astype(np.float64), scd)
        gg = g.cpu().numpy().astype(np.float64)
        assert np.abs(gg - gref).max() <= 1e-5 * np.abs(gref).max(), np.abs(gg - gref).max() / np.abs(gref).max()
        assert abs(float(loss.item()) - lref) <= 1e-5 * lref
    finally:
        fea.fea_costmodel_destroy(h)


def test_adam_steps_and_inference_match_oracle():
    import torch
    fea = engine()
    X, y = _data(3000, seed=5)
    p0 = M.xavier_init(6).astype(np.float32)
    h = fea.fea_costmodel_create(6, p0)
    try:
        Xd, yd = _tensors(X, y)
        fea.fea_costmodel_fit_scaler(h, Xd, yd)
        _, sc = fea.fea_costmodel_get_params(h, 6)
        scd = (sc[:6].astype(np.float64), sc[6:12].astype(np.float64), float(sc[12]), float(sc[13]))
        # three Adam steps, each checked against the oracle update driven by the GPU's own gradient
        p = p0.astype(np.float64); m = np.zeros_like(p); v = np.zeros_like(p)
        lr = 1e-2
        for k in range(1, 4):
            g, _ = fea.fea_costmodel_grad(h, Xd, yd, 1313)
            fea.fea_costmodel_train(h, Xd, yd, 1, lr)
            p, m, v = M.adam_step(p, m, v, g.cpu().numpy().astype(np.float64), k, lr)
            pg, _ = fea.fea_costmodel_get_params(h, 6)
            assert np.abs(pg - p).max() <= 1e-5 * lr * k + 1e-6 * np.abs(p).max()
        # then train and compare predictions at the GPU's parameters
        loss = fea.fea_costmodel_train(h, Xd, yd, 400, lr)
        pg, _ = fea.fea_costmodel_get_params(h, 6)
        pred = fea.fea_costmodel_predict(h, Xd).cpu().numpy()
        ref = M.predict(pg.astype(np.float64), 6, scd, X.astype(np.float64))
        assert np.abs(pred - ref).max() <= 1e-5 * np.abs(ref).max()
        # the model learned the synthetic cost law (standardised MSE well below 1)
        assert float(loss.item()) < 0.05
    finally:
        fea.fea_costmodel_destroy(h)


def test_item_features_match_oracle():
    import torch
    fea = engine()
    mesh = mg.hybrid_cube(4, 5)
    rng = np.random.default_rng(3)
    state = np.zeros((mesh.n_elems, 8, 7)); state[:, :, 6] = rng.uniform(-1, 1, (mesh.n_elems, 8)).clip(0)
    U = mg.fourier_displacement(mesh.coords, 1e-4, seed=4)
    s = fea.System.from_mesh(mesh, 3)
    try:
        for chunk in (1, 7, 0):
            t, f, c = fea.fea_work_items(s.handle, chunk)
            X = fea.fea_item_features(s.handle, chunk, len(t), torch.tensor(U.reshape(-1), device="cuda"),
                                      torch.tensor(state, device="cuda")).cpu().numpy()
            ref = M.item_features(mesh, chunk if chunk else 128, U, state)
            np.testing.assert_array_equal(X[:, :4], ref[:, :4])
            np.testing.assert_allclose(X[:, 4], ref[:, 4], rtol=1e-6, atol=1e-7)
            np.testing.assert_allclose(X[:, 5], ref[:, 5], rtol=1e-5)
    finally:
        s.close()


def _time_assemble(s, op, reps=7):
    import torch
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        s.assemble(op)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    s.check()
    return float(np.median(ts))


def test_mlp_packing_makespan_against_gauss_point_weights_and_stealing(capsys):
    """The learned model packs the J2 work items at least as well as the
    Gauss-point-weight heuristic (the paper's a-priori element weight);
    dynamic work stealing is the reference makespan."""
    import json
    import os
    import torch
    fea = engine()
    amp = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "j2_amplitude.json")))["amplitude"]
    mesh, U = mg.j2_workload(40, amp)
    s = fea.System.from_mesh(mesh, 3)
    try:
        u = torch.tensor(U.reshape(-1), device="cuda")
        st1 = torch.empty((mesh.n_elems, 8, 7), dtype=torch.float64, device="cuda")
        s.assemble(fea.make_operator(kind=fea.FEA_OP_J2, precision=1, u=0.5 * u, state_out=st1))
        chunk = 32
        types, _, counts = fea.fea_work_items(s.handle, chunk)
        n_items = len(counts)
        item_ns = torch.zeros(n_items, dtype=torch.int64, device="cuda")
        base = dict(kind=fea.FEA_OP_J2, precision=1, u=u, state_in=st1, chunk=chunk)
        steal = fea.make_operator(schedule=fea.FEA_SCHED_STEAL, item_ns=item_ns, **base)
        t_steal = _time_assemble(s, steal)
        # training data: the per-item timings the assembly recorded
        X = fea.fea_item_features(s.handle, chunk, n_items, u, st1)
        y = torch.log(item_ns.to(torch.float32) / torch.tensor(counts, device="cuda", dtype=torch.float32))
        h = fea.fea_costmodel_create(6, M.xavier_init(6).astype(np.float32))
        try:
            fea.fea_costmodel_fit_scaler(h, X, y)
            loss = float(fea.fea_costmodel_train(h, X, y, 600, 1e-2).item())
            pred = fea.fea_costmodel_predict(h, X).cpu().numpy().astype(np.float64)
        finally:
            fea.fea_costmodel_destroy(h)
        grid = fea.fea_persistent_grid(steal, s.handle)
        cost_mlp = np.exp(pred) * counts
        cost_gp = counts * np.array([4, 8, 6, 8])[types].astype(np.float64)
        res = {}
        for name, cost in (("mlp", cost_mlp), ("gauss_points", cost_gp)):
            q, off, _ = fea.fea_pack_lpt(cost, grid)
            qd, od = torch.tensor(q, device="cuda"), torch.tensor(off, device="cuda")
            op = fea.make_operator(schedule=fea.FEA_SCHED_QUEUES, n_ctas=grid, queue=qd, queue_off=od, **base)
            res[name] = _time_assemble(s, op)
        with capsys.disabled():
            print(f"\nJ2 40^3 chunk {chunk}: {n_items} items on {grid} CTAs; train loss {loss:.3f}; "
                  f"makespan ms: steal {t_steal:.3f}, mlp {res['mlp']:.3f}, gauss-point {res['gauss_points']:.3f}")
        assert loss < 1.0
        assert res["mlp"] <= 1.02 * res["gauss_points"]
    finally:
        s.close()
