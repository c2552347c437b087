"""The bench's algorithmic work counts (the roofline numerators), pinned on CPU.

* Accumulation adds and bytes: brute force over the elements and arrays of
  small tet, hex, hybrid and batch-style meshes.
* Per-element flops: an element routine written with an operation-counting
  number type follows the algorithm each count describes (modal hex
  Jacobian, affine tets, isoparametric pyramids and prisms; FP64 geometry,
  FP32 integration) and must reproduce the oracle's element matrix and right
  hand side -- so the counted algorithm computes the right thing -- while
  doing exactly the operations ``bench.element_flops`` states.
"""
import math

import numpy as np
import pytest

import bench
from paper_1805_03949_gb300 import meshgen as mg

# ---------------------------------------------------------------------------
# counting numbers: + - * / sqrt count 1, fma 2; sign flips are free
# ---------------------------------------------------------------------------

COUNT = {}
ROLE = ["geometry"]


def _v(x):
    return x.v if isinstance(x, Num) else float(x)


def _tick(n=1):
    COUNT[ROLE[0]] = COUNT.get(ROLE[0], 0) + n


class Num:
    __slots__ = ("v",)

    def __init__(self, v):
        self.v = float(v)

    def __add__(self, o):
        _tick(); return Num(self.v + _v(o))

    __radd__ = __add__

    def __sub__(self, o):
        _tick(); return Num(self.v - _v(o))

    def __rsub__(self, o):
        _tick(); return Num(_v(o) - self.v)

    def __mul__(self, o):
        _tick(); return Num(self.v * _v(o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        _tick(); return Num(self.v / _v(o))

    def __rtruediv__(self, o):
        _tick(); return Num(_v(o) / self.v)

    def __neg__(self):
        return Num(-self.v)


def fma(a, b, c):
    _tick(2)
    return Num(_v(a) * _v(b) + _v(c))


def sqrt(a):
    _tick()
    return Num(math.sqrt(_v(a)))


def _dot_acc(terms, acc=0.0):
    """sum of products as a chain of FMAs from acc"""
    for x, y in terms:
        acc = fma(x, y, acc)
    return acc


def _cofactors(J):
    C = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            i1, i2 = sorted({0, 1, 2} - {i})
            j1, j2 = sorted({0, 1, 2} - {j})
            sgn = -1.0 if (i + j) % 2 else 1.0
            m = fma(J[i1][j1], J[i2][j2], -(J[i1][j2] * J[i2][j1]))   # 1 mul + 1 FMA
            C[i][j] = -m if sgn < 0 else m
    return C


def _det(J, C):
    return fma(J[0][2], C[0][2], fma(J[0][1], C[0][1], J[0][0] * C[0][0]))  # 1 mul + 2 FMA


HEX_BITS = [0, 1, 3, 2, 4, 5, 7, 6]   # binary corner p -> local VTK node (the engine's order)


def counted_element(O, etype, X, op, tet_rule, k0=1.0, k2=0.0, f=(1.0, 1.0, 1.0), young=1.0, nu=0.3):
    """Element matrix and RHS by the counted algorithm; returns (A, b, counts by role)."""
    COUNT.clear()
    nn = bench.NODES_PER_TYPE[etype]
    d = 1 if op == bench.OP_DIFFUSION else 3
    pts, w = O.quadrature(etype, tet_rule)
    nq = len(w)
    k_varies = op == bench.OP_DIFFUSION and k2 != 0.0
    lam = young * nu / ((1 + nu) * (1 - 2 * nu))
    mu = young / (2 * (1 + nu))
    Xn = [[Num(x) for x in row] for row in np.asarray(X)]
    ROLE[0] = "geometry"
    shapes = [O.shape(etype, p) for p in pts]
    # ---- geometry (FP64): J, C, det J, w det J per point; gradient scale
    per_point = []   # (C, det-factor, wdet) per point
    if etype == 3:
        g = 1.0 / math.sqrt(3.0)
        # modal coefficients: 3 Walsh-Hadamard stages on the corners (binary order)
        v = [[Xn[HEX_BITS[p]][i] for i in range(3)] for p in range(8)]
        for s in range(3):
            bit = 1 << s
            v = [[(v[p][i] - v[p ^ bit][i]) if p & bit else (v[p][i] + v[p ^ bit][i]) for i in range(3)]
                 for p in range(8)]
        hex_pts = [((1 if q & 1 else -1) * g, (1 if q & 2 else -1) * g, (1 if q & 4 else -1) * g) for q in range(8)]
        shapes = [O.shape(3, p) for p in hex_pts]
        wq = [1.0] * 8
        # column c of J depends only on the other two point coordinates: each
        # of its 4 distinct values is formed once and shared by two points
        cols = [{}, {}, {}]

        def column(c, s, t):
            if (s, t) not in cols[c]:
                if c == 0:    # (y, z)
                    cols[c][(s, t)] = [fma(v[7][i], s * t, fma(v[5][i], t, fma(v[3][i], s, v[1][i]))) for i in range(3)]
                elif c == 1:  # (x, z)
                    cols[c][(s, t)] = [fma(v[7][i], s * t, fma(v[6][i], t, fma(v[3][i], s, v[2][i]))) for i in range(3)]
                else:         # (x, y)
                    cols[c][(s, t)] = [fma(v[7][i], s * t, fma(v[6][i], t, fma(v[5][i], s, v[4][i]))) for i in range(3)]
            return cols[c][(s, t)]

        for q, (x, y, z) in enumerate(hex_pts):
            c0, c1, c2 = column(0, y, z), column(1, x, z), column(2, x, y)
            J = [[c0[i], c1[i], c2[i]] for i in range(3)]
            C = _cofactors(J)
            det = _det(J, C)                       # det J' = 512 det J
            wdet = wq[q] * det * (1.0 / 512.0)     # 2 mul
            per_point.append((C, det, wdet, 8.0))
        nq, w = 8, wq
    elif etype == 0:
        E = [[Xn[a][i] - Xn[0][i] for a in (1, 2, 3)] for i in range(3)]   # J_ij = x_j - x_0 (9 subs)
        C = _cofactors(E)
        det = _det(E, C)
        inv = 1.0 / det
        for q in range(nq):
            per_point.append((C, inv, w[q] * det, None))
    else:
        D = [[Xn[a][i] - Xn[0][i] for i in range(3)] for a in range(1, nn)]   # 3 (nn - 1) subs
        for q in range(nq):
            dN = shapes[q][1]
            J = [[_dot_acc([(D[a - 1][i], dN[a][j]) for a in range(1, nn)]) for j in range(3)] for i in range(3)]
            C = _cofactors(J)
            det = _det(J, C)
            per_point.append((C, det, w[q] * det, None))
    # x_q for k(x) (FP64 coordinates)
    xq = []
    if k_varies:
        ROLE[0] = "coords"
        for q in range(nq):
            N = shapes[q][0]
            xq.append(_dot_acc([(N[a], Xn[a][0]) for a in range(nn)]))
    # ---- integration (FP32 in FP32-integrate)
    ROLE[0] = "integrate"
    A = [[Num(0.0) for _ in range(nn * d)] for _ in range(nn * d)]
    b = [Num(0.0) for _ in range(nn * d)]

    def grads(q, scaled):
        C, det, wdet, jscale = per_point[q]
        dN = shapes[q][1]
        if scaled:
            s = sqrt(wdet) * jscale / det if jscale else sqrt(wdet) * (1.0 / det)   # 3 ops
        else:
            s = det                                    # affine: 1/det J, taken once with the geometry
        out = []
        for a in range(nn):
            out.append([_dot_acc([(C[i][j], dN[a][j]) for j in range(3)]) * s for i in range(3)])
        return out

    if etype == 0:
        G = grads(0, False)           # constant gradients, once
        Wk = Num(0.0)
        for q in range(nq):
            kq = k0 if not k_varies else fma(k2 * xq[q], xq[q], k0)
            Wk = fma(per_point[q][2], kq, Wk)
        if op == bench.OP_DIFFUSION:
            for a in range(nn):
                for bb in range(a, nn):
                    A[a][bb] = Wk * _dot_acc([(G[a][i], G[bb][i]) for i in range(3)])
        else:
            lw, mw = lam * Wk, mu * Wk
            M = {}
            _moments(M, G, nn)
            _elastic_blocks(A, M, lw, mw, nn)
    else:
        M = {}
        for q in range(nq):
            G = grads(q, True)
            if op == bench.OP_DIFFUSION:
                kq = Num(k0) if not k_varies else fma(k2 * xq[q], xq[q], k0)
                kG = [[kq * G[a][i] for i in range(3)] for a in range(nn)]
                for a in range(nn):
                    for bb in range(a, nn):
                        A[a][bb] = _dot_acc([(kG[a][i], G[bb][i]) for i in range(3)], A[a][bb])
            else:
                _moments(M, G, nn)
        if op != bench.OP_DIFFUSION:
            _elastic_blocks(A, M, lam, mu, nn)
    for q in range(nq):
        N = shapes[q][0]
        wdet = per_point[q][2]
        for a in range(nn):
            for c in range(d):
                b[d * a + c] = fma(wdet, N[a] * f[c], b[d * a + c])
    # symmetric fill (no arithmetic)
    An = np.zeros((nn * d, nn * d))
    for r in range(nn * d):
        for c in range(nn * d):
            An[r, c] = A[r][c].v
    if op == bench.OP_DIFFUSION:
        An = np.triu(An) + np.triu(An, 1).T
    else:
        for a in range(nn):
            for bb in range(a + 1, nn):
                An[3 * bb:3 * bb + 3, 3 * a:3 * a + 3] = An[3 * a:3 * a + 3, 3 * bb:3 * bb + 3].T
    return An, np.array([x.v for x in b]), dict(COUNT), nq


def _moments(M, G, nn):
    """M_ab += g_a g_b^T for a <= b (9 FMA per block)."""
    for a in range(nn):
        for bb in range(a, nn):
            m = M.setdefault((a, bb), [[Num(0.0)] * 3 for _ in range(3)])
            for i in range(3):
                for j in range(3):
                    m[i][j] = fma(G[a][i], G[bb][j], m[i][j])


def _elastic_blocks(A, M, lam, mu, nn):
    """A_ab = lam M_ab + mu M_ab^T + mu tr(M_ab) I for a <= b (33 per block)."""
    for a in range(nn):
        for bb in range(a, nn):
            m = M[(a, bb)]
            mt = mu * (m[0][0] + m[1][1] + m[2][2])
            for i in range(3):
                for j in range(3):
                    A[3 * a + i][3 * bb + j] = fma(lam, m[i][j], mu * m[j][i])
                A[3 * a + i][3 * bb + i] = A[3 * a + i][3 * bb + i] + mt


CASES = [
    # etype, op, tet_rule, k2 (diffusion)
    (3, bench.OP_ELASTICITY, 1, 0.0),
    (3, bench.OP_DIFFUSION, 1, 1.0),
    (0, bench.OP_ELASTICITY, 1, 0.0),
    (0, bench.OP_DIFFUSION, 1, 1.0),
    (0, bench.OP_DIFFUSION, 0, 0.0),
    (1, bench.OP_DIFFUSION, 1, 1.0),
    (2, bench.OP_DIFFUSION, 1, 1.0),
    (2, bench.OP_ELASTICITY, 1, 0.0),
    (1, bench.OP_ELASTICITY, 1, 0.0),
]


def _element_coords(etype):
    mesh = {0: mg.template_cube(1, mg.TET4, 0.0), 1: mg.template_cube(1, mg.PYR5, 0.0),
            2: mg.template_cube(1, mg.PRISM6, 0.0), 3: mg.hex_cube(1, 0.0)}[etype]
    nn = bench.NODES_PER_TYPE[etype]
    X = mesh.coords[mesh.conn[:nn]].copy()
    rng = np.random.default_rng(etype + 10)
    return X + rng.uniform(-0.05, 0.05, X.shape)


@pytest.mark.parametrize("etype,op,tet_rule,k2", CASES)
def test_element_flops_count_an_algorithm_that_matches_the_oracle(oracle, etype, op, tet_rule, k2):
    X = _element_coords(etype)
    kw = dict(k0=1.0, k2=k2, source=1.0) if op == bench.OP_DIFFUSION else dict(young=1.0, poisson=0.3)
    Ae, be, _, _ = oracle.element(etype, X, op, tet_rule, **kw)
    A, b, counts, nq = counted_element(oracle, etype, X, op, tet_rule, k0=1.0, k2=k2)
    scale = np.abs(Ae).max()
    assert np.max(np.abs(A - Ae)) <= 1e-12 * scale
    assert np.max(np.abs(b - be)) <= 1e-12 * np.abs(be).max()
    w = bench.element_flops(etype, op, nq, k_varies=k2 != 0.0)
    assert counts.get("geometry", 0) == w["geometry"], (counts, w)
    assert counts.get("coords", 0) == w["coords"], (counts, w)
    assert counts.get("integrate", 0) == w["grad"] + w["prod"] + w["rhs"], (counts, w)


# ---------------------------------------------------------------------------
# accumulation adds and bytes: brute force
# ---------------------------------------------------------------------------

def _brute(mesh, d):
    """(c - 1) FP64 adds per upper entry of A with c contributions (i <= j node
    pairs, d x d each) and per b entry; bytes of A, b, coordinates, row starts,
    connectivity and the node map."""
    from oracle import oracle as O
    off = np.asarray(mesh.conn_offsets)
    conn = np.asarray(mesh.conn)
    contrib = {}
    bcount = np.zeros(mesh.n_nodes, dtype=np.int64)
    for e in range(mesh.n_elems):
        nodes = conn[off[e]:off[e + 1]]
        for a in nodes:
            bcount[a] += 1
            for bb in nodes:
                if a <= bb:
                    contrib[(int(a), int(bb))] = contrib.get((int(a), int(bb)), 0) + 1
    adds = d * d * sum(c - 1 for c in contrib.values()) + d * int((bcount - 1).clip(min=0).sum())
    rp, col, nmap = O.pattern(mesh, d)
    nn = np.diff(off)
    by = (8 * len(col) + 8 * d * mesh.n_nodes + 24 * mesh.n_nodes + 8 * d * mesh.n_nodes
          + 4 * int(nn.sum()) + 4 * len(nmap))
    return adds, by, len(col) // (d * d)


@pytest.mark.parametrize("name,d", [("kuhn3", 1), ("hybrid2", 1), ("hybrid2", 3), ("hex3", 3), ("tet_box", 3)])
def test_accumulation_and_bytes_match_brute_force(name, d):
    mesh = {"kuhn3": lambda: mg.kuhn_tet_cube(3), "hybrid2": lambda: mg.hybrid_cube(2, 11),
            "hex3": lambda: mg.hex_cube(3, 0.2, 2), "tet_box": lambda: mg.template_cube(2, mg.TET4, 0.2, 3)}[name]()
    adds, by, nnz_node = _brute(mesh, d)
    counts = {t: int(c) for t, c in enumerate(np.bincount(mesh.types, minlength=4)) if c}
    op = bench.OP_DIFFUSION if d == 1 else bench.OP_ELASTICITY
    w = bench.assembly_work(counts, mesh.n_nodes, nnz_node, op, 1)
    assert w["parts"]["accumulate"] == adds
    assert w["bytes"] == by


def test_j2_bytes_add_displacements_and_state():
    mesh = mg.hex_cube(2, 0.2, 2)
    _, by, nnz_node = _brute(mesh, 3)
    w = bench.assembly_work({3: mesh.n_elems}, mesh.n_nodes, nnz_node, bench.OP_J2, 1,
                            j2={"points": 64, "plastic_points": 10, "newton_iters": 25})
    assert w["bytes"] == by + 24 * mesh.n_nodes + mesh.n_elems * 2 * 8 * 7 * 8
    base = bench.assembly_work({3: mesh.n_elems}, mesh.n_nodes, nnz_node, bench.OP_ELASTICITY, 1)
    # the J2 update: per point, more per plastic point and per Newton iteration (FP64 in both precisions)
    assert w["parts"]["j2_update"] == (64 * bench.j2_point_flops(False, 0)
                                       + 10 * (bench.j2_point_flops(True, 0) - bench.j2_point_flops(False, 0))
                                       + 20 * 25)
    assert w["fp64"] == base["fp64"] + 72 * mesh.n_elems + w["parts"]["j2_update"]


def test_step_roofline_picks_the_binding_resource():
    peaks = {"fp64": 1e12, "fp32": 50e12, "hbm": 5e12}
    r = bench.step_roofline({"fp64": 2e9, "fp32": 10e9, "bytes": 5e9}, 4.0, peaks)
    assert r["resource"] == "fp64" and r["t_roof_ms"] == pytest.approx(2.0) and r["frac"] == pytest.approx(0.5)
    r = bench.step_roofline({"fp64": 1e8, "fp32": 1e9, "bytes": 5e9}, 2.0, peaks)
    assert r["resource"] == "hbm" and r["bound"] == "hbm" and r["frac"] == pytest.approx(0.5)
