"""Pins of the cost-model, feature and packing oracle (CPU only): finite
differences, closed forms, brute force and exact properties.
"""
import itertools

import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_1805_03949_gb300 import meshgen as mg


def _data(n=200, n_in=6, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n_in)) * np.array([1, 2, 3, 0.5, 1e-3, 10][:n_in]) + 4.0
    y = np.sin(X[:, 0]) + 0.1 * X[:, 1] + rng.normal(size=n) * 0.05
    return X, y


def test_parameter_count_and_layout():
    assert M.n_params(6) == 1313
    p = mg.mlp_initial_params(6)
    parts = M.unpack(p, 6)
    assert [np.size(x) for x in parts] == [192, 32, 1024, 32, 32, 1]
    np.testing.assert_array_equal(M.pack(*parts), p)
    # Xavier-uniform bounds, zero biases
    assert np.abs(parts[0]).max() <= np.sqrt(6 / 38) and np.abs(parts[2]).max() <= np.sqrt(6 / 64)
    assert not parts[1].any() and not parts[3].any() and parts[5] == 0.0


def test_scaler_standardises_and_guards_constant_columns():
    X, y = _data()
    X[:, 3] = 7.0                                     # a constant feature
    xm, xs, ym, ys = M.fit_scaler(X, y)
    Xs = (X - xm) / xs
    np.testing.assert_allclose(Xs[:, [0, 1, 2, 4, 5]].mean(axis=0), 0, atol=1e-10)
    np.testing.assert_allclose(Xs[:, [0, 1, 2, 4, 5]].std(axis=0), 1, rtol=1e-12)
    assert xs[3] == 1.0 and np.all(Xs[:, 3] == 0)


def test_forward_closed_form():
    """With zero hidden weights the output is b3 + w3 . tanh(b2), independent of x."""
    W1 = np.zeros((32, 6)); W2 = np.zeros((32, 32))
    b1 = np.linspace(-1, 1, 32); b2 = np.linspace(0.5, -0.5, 32); w3 = np.linspace(-2, 2, 32)
    p = M.pack(W1, b1, W2, b2, w3, 0.25)
    out, H1, _ = M.forward(p, 6, np.random.default_rng(0).normal(size=(5, 6)))
    np.testing.assert_allclose(out, 0.25 + w3 @ np.tanh(b2), rtol=1e-15)
    np.testing.assert_allclose(H1, np.tile(np.tanh(b1), (5, 1)), rtol=1e-15)


def test_predict_undoes_the_standardisation():
    """On the training data, the mean squared error of the predictions in
    target units is the standardised loss times the target variance, and a
    network whose last layer is zero predicts the target mean."""
    X, y = _data()
    sc = M.fit_scaler(X, y)
    p = mg.mlp_initial_params(6, seed=8)
    loss, _ = M.loss_grad(p, 6, X, y, sc)
    pred = M.predict(p, 6, sc, X)
    assert np.mean((pred - y) ** 2) == pytest.approx(loss * sc[3] ** 2, rel=1e-12)
    W1, b1, W2, b2, w3, b3 = M.unpack(p, 6)
    zero = M.pack(W1, b1, W2, b2, np.zeros_like(w3), 0.0)
    np.testing.assert_allclose(M.predict(zero, 6, sc, X), np.full(len(y), y.mean()), rtol=1e-14)


def test_gradient_matches_central_differences():
    X, y = _data(60)
    p = mg.mlp_initial_params(6) + np.random.default_rng(3).normal(size=1313) * 0.05
    sc = M.fit_scaler(X, y)
    _, g = M.loss_grad(p, 6, X, y, sc)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(1313, 60, replace=False), [0, 191, 192, 223, 1247, 1280, 1311, 1312]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p); e[i] = h
        fd = (M.loss_grad(p + e, 6, X, y, sc)[0] - M.loss_grad(p - e, 6, X, y, sc)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, np.abs(g).max()), (i, fd, g[i])


def test_first_adam_step_is_minus_lr_sign():
    """Bias correction makes the first step -lr * g / (|g| + eps)."""
    g = np.array([3.0, -0.5, 1e-3, -2e-2])
    p, m, v = M.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_training_decreases_the_loss():
    X, y = _data(300)
    p0 = mg.mlp_initial_params(6)
    _, sc, losses = M.train(p0, 6, X, y, 200, 1e-2)
    assert losses[-1] < 0.2 * losses[0]


def _brute_makespan(costs, m):
    best = np.inf
    for assign in itertools.product(range(m), repeat=len(costs)):
        loads = np.zeros(m)
        for c, q in zip(costs, assign):
            loads[q] += c
        best = min(best, loads.max())
    return best


@pytest.mark.parametrize("seed", range(6))
def test_lpt_properties_and_graham_bound(seed):
    rng = np.random.default_rng(seed)
    n, m = 7, 2 + seed % 2
    costs = rng.uniform(1, 10, n).round(3)
    ids, off, loads = M.lpt(costs, m)
    assert sorted(ids.tolist()) == list(range(n))                 # every item exactly once
    for q in range(m):
        np.testing.assert_allclose(costs[ids[off[q]:off[q + 1]]].sum(), loads[q])
    # replay: each item went onto a least-loaded queue at its turn
    cur = np.zeros(m)
    owner = {int(i): q for q in range(m) for i in ids[off[q]:off[q + 1]]}
    for i in sorted(range(n), key=lambda i: (-costs[i], i)):
        assert cur[owner[i]] == cur.min()
        cur[owner[i]] += costs[i]
    opt = _brute_makespan(costs, m)
    assert loads.max() <= (4 / 3 - 1 / (3 * m)) * opt + 1e-9


@pytest.mark.parametrize("etype", [mg.TET4, mg.PYR5, mg.PRISM6, mg.HEX8])
def test_centroid_strain_is_exact_for_affine_displacements(etype):
    """u = G x has strain sym(G) everywhere, for any element shape."""
    mesh = mg.template_cube(2, etype, 0.2, 3)
    G = np.array([[1e-3, 2e-3, -1e-3], [4e-4, -2e-3, 5e-4], [3e-3, 1e-3, 2e-3]])
    U = mesh.coords @ G.T
    F = M.element_features(mesh, U)
    S = 0.5 * (G + G.T)
    np.testing.assert_allclose(F[:, 5], np.sqrt((S * S).sum()), rtol=1e-12)
    assert (F[:, etype] == 1).all() and F[:, :4].sum(axis=1).max() == 1


def test_item_features_average_their_elements():
    mesh = mg.hybrid_cube(3, 5)
    rng = np.random.default_rng(2)
    state = np.zeros((mesh.n_elems, 8, 7)); state[:, :, 6] = rng.uniform(-1, 1, (mesh.n_elems, 8)).clip(0)
    U = mg.fourier_displacement(mesh.coords, 1e-4, seed=4)
    items = M.work_items(mesh, 5)
    X = M.item_features(mesh, 5, U, state)
    assert sum(c for _, _, c in items) == mesh.n_elems and len(X) == len(items)
    F = M.element_features(mesh, U, state)
    t, f, c = items[3]
    ids = np.nonzero(mesh.types == t)[0][f:f + c]
    np.testing.assert_allclose(X[3], F[ids].mean(axis=0))
    nq = np.array([4, 8, 6, 8])[mesh.types]
    frac = np.array([(state[e, :nq[e], 6] > 0).mean() for e in range(mesh.n_elems)])
    np.testing.assert_allclose(F[:, 4], frac)
