"""Plain FP64 reference of the learned cost model and of the queue packing.

TEST INFRASTRUCTURE ONLY: used by the tests, never by the engine, and it
shares no code with it.  What it computes:

* the cost model: x (n_in features, standardised by the training set's mean
  and population standard deviation, a zero deviation replaced by 1) ->
  32 tanh -> 32 tanh -> 1 (standardised log nanoseconds per element); loss =
  mean squared error; Adam (Kingma and Ba, 2015: beta1 0.9, beta2 0.999,
  eps 1e-8, bias-corrected moments), full batch.  Parameter vector order:
  W1 [32][n_in], b1 [32], W2 [32][32], b2 [32], w3 [32], b3.
* the item features: per element, the one-hot type, the fraction of its
  Gauss points with a positive committed equivalent plastic strain, and the
  Frobenius norm of sym(grad u) at the reference centroid; per item (a run of
  `chunk` elements of one type in upload order), the mean over its elements.
* longest-processing-time-first packing (Graham, 1969): items in decreasing
  cost (ties: lower id first) onto the least-loaded queue (ties: lower queue).
"""
from __future__ import annotations

import heapq

import numpy as np

from . import oracle as _o

HID = 32


def n_params(n_in: int) -> int:
    """Length of the parameter vector for n_in features."""
    return HID * n_in + HID + HID * HID + HID + HID + 1


def unpack(p, n_in):
    """(W1, b1, W2, b2, w3, b3) views of the parameter vector, in FP64."""
    p = np.asarray(p, dtype=np.float64)
    k = 0
    W1 = p[k:k + HID * n_in].reshape(HID, n_in); k += HID * n_in
    b1 = p[k:k + HID]; k += HID
    W2 = p[k:k + HID * HID].reshape(HID, HID); k += HID * HID
    b2 = p[k:k + HID]; k += HID
    w3 = p[k:k + HID]; k += HID
    b3 = p[k]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    """The parameter vector of the six arrays, in their order."""
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [b3]])


def fit_scaler(X, y):
    """(x mean, x std, y mean, y std), population deviations; a zero deviation becomes 1."""
    X = np.asarray(X, dtype=np.float64); y = np.asarray(y, dtype=np.float64)
    xm = X.mean(axis=0); xs = X.std(axis=0)
    ym = y.mean(); ys = y.std()
    xs = np.where(xs > 1e-12 * (np.abs(xm) + 1e-30), xs, 1.0)
    ys = ys if ys > 1e-12 * (abs(ym) + 1e-30) else 1.0
    return xm, xs, ym, ys


def forward(p, n_in, Xs):
    """Network output for standardised inputs Xs [n, n_in]; returns (out, H1, H2)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in)
    H1 = np.tanh(Xs @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    return H2 @ w3 + b3, H1, H2


def loss_grad(p, n_in, X, y, scaler):
    """Mean squared error on standardised data and its gradient (backpropagation)."""
    xm, xs, ym, ys = scaler
    Xs = (np.asarray(X, dtype=np.float64) - xm) / xs
    t = (np.asarray(y, dtype=np.float64) - ym) / ys
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in)
    out, H1, H2 = forward(p, n_in, Xs)
    n = len(t)
    r = out - t
    loss = float((r * r).mean())
    d3 = 2.0 * r / n
    gw3 = H2.T @ d3
    gb3 = d3.sum()
    D2 = np.outer(d3, w3) * (1.0 - H2 * H2)
    gW2 = D2.T @ H1
    gb2 = D2.sum(axis=0)
    D1 = (D2 @ W2) * (1.0 - H1 * H1)
    gW1 = D1.T @ Xs
    gb1 = D1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gw3, gb3)


def adam_step(p, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update (step counts from 1)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def train(p, n_in, X, y, epochs, lr, scaler=None):
    """Full-batch Adam from p for `epochs` steps: (parameters, scaler, the
    loss of every epoch before its update)."""
    scaler = scaler or fit_scaler(X, y)
    m = np.zeros_like(p); v = np.zeros_like(p)
    losses = []
    for k in range(1, epochs + 1):
        loss, g = loss_grad(p, n_in, X, y, scaler)
        losses.append(loss)
        p, m, v = adam_step(p, m, v, g, k, lr)
    return p, scaler, losses


def predict(p, n_in, scaler, X):
    """Predictions in target units for the rows of X."""
    xm, xs, ym, ys = scaler
    out, _, _ = forward(p, n_in, (np.asarray(X, dtype=np.float64) - xm) / xs)
    return out * ys + ym


def lpt(costs, n_queues):
    """(queue ids, offsets [n_queues + 1], loads): greedy LPT, queues in assignment order."""
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, q) for q in range(n_queues)]
    owner = np.zeros(len(costs), dtype=np.int64)
    per_q = [[] for _ in range(n_queues)]
    for i in order:
        load, q = heapq.heappop(heap)
        owner[i] = q
        per_q[q].append(i)
        heapq.heappush(heap, (load + costs[i], q))
    loads = np.array([costs[per_q[q]].sum() if per_q[q] else 0.0 for q in range(n_queues)])
    off = np.concatenate([[0], np.cumsum([len(x) for x in per_q])])
    ids = np.array([i for x in per_q for i in x], dtype=np.int64)
    return ids, off, loads


def work_items(mesh, chunk=128):
    """(type, first, count) per item: per type in enum order, runs of chunk elements in upload order."""
    items = []
    for t in range(4):
        n = int((mesh.types == t).sum())
        for f in range(0, n, chunk):
            items.append((t, f, min(chunk, n - f)))
    return items


_CENTROIDS = {0: (0.25, 0.25, 0.25), 1: (0.0, 0.0, 0.25), 2: (1.0 / 3.0, 1.0 / 3.0, 0.0), 3: (0.0, 0.0, 0.0)}
_NQ = {0: 4, 1: 8, 2: 6, 3: 8}


def element_features(mesh, U=None, state=None):
    """[E, 6] per-element features (one-hot type, yielded fraction, centroid strain norm), FP64."""
    E = mesh.n_elems
    F = np.zeros((E, 6))
    F[np.arange(E), mesh.types] = 1.0
    off = mesh.conn_offsets
    for t in range(4):
        ids = np.nonzero(mesh.types == t)[0]
        if not len(ids):
            continue
        nn = _o.NODES[t]
        conn = np.stack([mesh.conn[off[ids] + a] for a in range(nn)], axis=1)   # [n, nn]
        if state is not None:
            F[ids, 4] = (np.asarray(state)[ids, :_NQ[t], 6] > 0).mean(axis=1)
        if U is not None:
            _, dN = _o.shape(t, _CENTROIDS[t])                                    # [nn, 3]
            X = mesh.coords[conn]                                                 # [n, nn, 3]
            J = np.einsum("eai,aj->eij", X - X[:, :1, :], dN)
            G = np.einsum("aj,eji->eai", dN, np.linalg.inv(J))                    # grad N_a = J^{-T} dN_a
            Gu = np.einsum("eai,eaj->eij", np.asarray(U)[conn], G)
            S = 0.5 * (Gu + np.transpose(Gu, (0, 2, 1)))
            F[ids, 5] = np.sqrt((S * S).sum(axis=(1, 2)))
    return F


def item_features(mesh, chunk=128, U=None, state=None):
    """Per work item (runs of `chunk` elements of one type), the mean of its elements' features."""
    F = element_features(mesh, U, state)
    out = []
    for t, f, c in work_items(mesh, chunk):
        ids = np.nonzero(mesh.types == t)[0][f:f + c]
        out.append(F[ids].mean(axis=0))
    return np.array(out)
