"""Pins of the FP64 CPU oracle against facts fixed by mathematics (no GPU).

The paper (Alg. "sequential assembly", Sec. 2.1.1) fixes the assembly loop but
prints no element formulation and no worked numbers, so the oracle is pinned
by closed forms: exact quadrature of monomials, shape-function identities,
exact rational element matrices, the Kuhn-lattice P1 stencil, the patch test,
rigid-body modes, zero row sums, symmetry, volume sums and brute-force
patterns on tiny meshes.  Each pin is chosen so that a dropped term, a sign
error, a transposed Jacobian or a wrong index fails at least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1805_03949_gb300 import meshgen as mg

REF_VOLUME = {mg.TET4: 1.0 / 6.0, mg.PYR5: 4.0 / 3.0, mg.PRISM6: 1.0, mg.HEX8: 8.0}
REF_NODES = {
    mg.TET4: [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)],
    mg.PYR5: [(-1, -1, 0), (1, -1, 0), (1, 1, 0), (-1, 1, 0), (0, 0, 1)],
    mg.PRISM6: [(0, 0, -1), (1, 0, -1), (0, 1, -1), (0, 0, 1), (1, 0, 1), (0, 1, 1)],
    mg.HEX8: [(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1),
              (-1, -1, 1), (1, -1, 1), (1, 1, 1), (-1, 1, 1)],
}


def _interior_points(etype, rng, n=20):
    pts = []
    while len(pts) < n:
        p = rng.uniform(-1, 1, 3)
        if etype == mg.TET4:
            p = rng.uniform(0, 1, 3)
            if p.sum() >= 0.98:
                continue
        elif etype == mg.PRISM6:
            p[:2] = rng.uniform(0, 1, 2)
            if p[0] + p[1] >= 0.98:
                continue
        elif etype == mg.PYR5:
            p[2] = rng.uniform(0.01, 0.95)
            if max(abs(p[0]), abs(p[1])) >= 1 - p[2]:
                continue
        pts.append(p)
    return pts


# ----------------------------------------------------------------------------
# quadrature
# ----------------------------------------------------------------------------

def _exact_monomial(etype, a, b, c):
    """Exact integral of x^a y^b z^c over the reference element."""
    f = math.factorial
    if etype == mg.TET4:
        return Fraction(f(a) * f(b) * f(c), f(a + b + c + 3))
    one_d = lambda k: Fraction(0) if k % 2 else Fraction(2, k + 1)
    if etype == mg.HEX8:
        return one_d(a) * one_d(b) * one_d(c)
    if etype == mg.PRISM6:
        return Fraction(f(a) * f(b), f(a + b + 2)) * one_d(c)
    # pyramid |x|,|y| <= 1 - z, z in [0,1]
    if a % 2 or b % 2:
        return Fraction(0)
    return Fraction(4, (a + 1) * (b + 1)) * Fraction(f(c) * f(a + b + 2), f(a + b + c + 3))


@pytest.mark.parametrize("etype,rule,deg", [(mg.TET4, 0, 1), (mg.TET4, 1, 2), (mg.PYR5, 1, 3),
                                            (mg.PRISM6, 1, 2), (mg.HEX8, 1, 3)])
def test_quadrature_exact_for_polynomials(oracle, etype, rule, deg):
    pts, w = oracle.quadrature(etype, rule)
    assert abs(w.sum() - REF_VOLUME[etype]) < 1e-15 * REF_VOLUME[etype]
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                q = float(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c))
                assert abs(q - float(_exact_monomial(etype, a, b, c))) < 1e-14, (a, b, c)


def test_quadrature_hex_tensor_degree3(oracle):
    pts, w = oracle.quadrature(mg.HEX8, 1)
    for a in range(4):
        for b in range(4):
            for c in range(4):
                q = float(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c))
                assert abs(q - float(_exact_monomial(mg.HEX8, a, b, c))) < 1e-14


def test_tet_four_point_rule_is_not_one_point(oracle):
    pts, w = oracle.quadrature(mg.TET4, 1)
    assert len(w) == 4 and not np.allclose(pts, 0.25)


# ----------------------------------------------------------------------------
# shape functions
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("etype", [mg.TET4, mg.PYR5, mg.PRISM6, mg.HEX8])
def test_shape_kronecker_unity_linear_reproduction(oracle, etype):
    nodes = np.array(REF_NODES[etype], dtype=np.float64)
    for a, p in enumerate(nodes):
        if etype == mg.PYR5 and a == 4:
            p = np.array([0.0, 0.0, 1.0 - 1e-9])
        N, _ = oracle.shape(etype, p)
        e = np.zeros(len(nodes)); e[a] = 1.0
        assert np.allclose(N, e, atol=1e-8)
    rng = np.random.default_rng(0)
    for p in _interior_points(etype, rng):
        N, dN = oracle.shape(etype, p)
        assert abs(N.sum() - 1.0) < 1e-14
        assert np.allclose(N @ nodes, p, atol=1e-14)          # x = sum N_a x_a reproduces xi
        assert np.allclose(dN.sum(axis=0), 0.0, atol=1e-14)
        assert np.allclose(dN.T @ nodes, np.eye(3), atol=1e-13)  # gradient of the identity map


@pytest.mark.parametrize("etype", [mg.TET4, mg.PYR5, mg.PRISM6, mg.HEX8])
def test_shape_derivatives_match_finite_differences(oracle, etype):
    rng = np.random.default_rng(1)
    h = 1e-6
    for p in _interior_points(etype, rng, 10):
        _, dN = oracle.shape(etype, p)
        for j in range(3):
            e = np.zeros(3); e[j] = h
            fd = (oracle.shape(etype, p + e)[0] - oracle.shape(etype, p - e)[0]) / (2 * h)
            assert np.allclose(dN[:, j], fd, atol=1e-8), (p, j)


# ----------------------------------------------------------------------------
# element matrices against exact rational integration
# ----------------------------------------------------------------------------

def _voigt_D(E, nu):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu)); mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] = lam + 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    return D


def _sym_box_hex_matrices(hx, hy, hz):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    signs = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    lin = lambda t, s, h: (t / h) if s else (1 - t / h)
    N = [lin(x, a, hx) * lin(y, b, hy) * lin(z, c, hz) for a, b, c in signs]
    G = [[sp.diff(n, v) for v in (x, y, z)] for n in N]
    box = ((x, 0, hx), (y, 0, hy), (z, 0, hz))
    GG = np.empty((8, 8, 3, 3), dtype=object)
    for a in range(8):
        for b in range(a, 8):
            for c in range(3):
                for cc in range(3):
                    GG[a, b, c, cc] = sp.integrate(sp.expand(G[a][c] * G[b][cc]), *box)
                    GG[b, a, cc, c] = GG[a, b, c, cc]
    NI = [sp.integrate(n, *box) for n in N]
    return GG.astype(float), np.array([float(v) for v in NI])


def test_hex8_box_matches_exact_integration(oracle):
    sp = pytest.importorskip("sympy")
    hx, hy, hz = sp.Rational(1, 3), sp.Rational(1, 5), sp.Rational(2, 7)
    GG, NI = _sym_box_hex_matrices(hx, hy, hz)
    X = np.array([(a * float(hx) + 0.3, b * float(hy) - 0.1, c * float(hz) + 2.0)
                  for a, b, c in [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                                  (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]])
    # diffusion, k = 1
    Ae, be, _, _ = oracle.element(mg.HEX8, X, oracle.OP_DIFFUSION, k0=1.0, k2=0.0, source=2.5)
    exact = np.einsum("abcc->ab", GG)
    assert np.allclose(Ae, exact, rtol=0, atol=1e-14 * np.abs(exact).max())
    assert np.allclose(be, 2.5 * NI, rtol=1e-14, atol=0)
    # elasticity: K_(a,c)(b,c') = lam G_ac G_bc' + mu G_ac' G_bc + mu delta_cc' G_a.G_b
    E, nu = 1.7, 0.27
    lam = E * nu / ((1 + nu) * (1 - 2 * nu)); mu = E / (2 * (1 + nu))
    Ke, fe, _, _ = oracle.element(mg.HEX8, X, oracle.OP_ELASTICITY, young=E, poisson=nu,
                                  body_force=(1.0, -2.0, 0.5))
    K = np.zeros((24, 24))
    for a in range(8):
        for b in range(8):
            for c in range(3):
                for cc in range(3):
                    v = lam * GG[a, b, c, cc] + mu * GG[a, b, cc, c]
                    if c == cc:
                        v += mu * np.trace(GG[a, b])
                    K[3 * a + c, 3 * b + cc] = v
    assert np.allclose(Ke, K, rtol=0, atol=1e-13 * np.abs(K).max())
    assert np.allclose(fe.reshape(8, 3), NI[:, None] * np.array([1.0, -2.0, 0.5]), rtol=1e-14)


def test_prism6_right_prism_matches_exact_integration(oracle):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    H = sp.Rational(3, 4)
    L = [1 - x - y, x, y]
    N = [L[i] * (1 - z / H) for i in range(3)] + [L[i] * (z / H) for i in range(3)]
    G = [[sp.diff(n, v) for v in (x, y, z)] for n in N]
    exact = np.zeros((6, 6))
    for a in range(6):
        for b in range(6):
            e = sp.expand(sum(G[a][c] * G[b][c] for c in range(3)))
            exact[a, b] = float(sp.integrate(e, (y, 0, 1 - x), (x, 0, 1), (z, 0, H)))
    X = np.array([(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 0.75), (1, 0, 0.75), (0, 1, 0.75)], dtype=float)
    Ae, _, _, _ = oracle.element(mg.PRISM6, X, oracle.OP_DIFFUSION, k0=1.0, k2=0.0)
    assert np.allclose(Ae, exact, rtol=0, atol=1e-14 * np.abs(exact).max())


def _sym_ref_pyramid_tensors():
    """Exact T[a, b, p, q] = int dN_a/dxi_p dN_b/dxi_q and NI[a] = int N_a over
    the reference pyramid (base [-1,1]^2 at zeta = 0, apex (0,0,1)), for the
    rational basis N_a = 1/4 [(1 + s_a x)(1 + t_a y) - z + s_a t_a x y z / (1 - z)],
    N_5 = z (Bedrosian 1992).  The collapsed map x = u (1 - z), y = v (1 - z)
    (volume factor (1 - z)^2) makes every integrand a polynomial in (u, v, z)."""
    sp = pytest.importorskip("sympy")
    x, y, z, u, v = sp.symbols("x y z u v")
    base = [(-1, -1), (1, -1), (1, 1), (-1, 1)]
    N = [sp.Rational(1, 4) * ((1 + s * x) * (1 + t * y) - z + s * t * x * y * z / (1 - z)) for s, t in base] + [z]
    G = [[sp.diff(n, w) for w in (x, y, z)] for n in N]
    sub = {x: u * (1 - z), y: v * (1 - z)}
    box = [(u, -1, 1), (v, -1, 1), (z, 0, 1)]

    def integral(f):
        return sp.integrate(sp.expand(sp.cancel(f.subs(sub) * (1 - z) ** 2)), *box)

    T = np.zeros((5, 5, 3, 3))
    for a in range(5):
        for b in range(a, 5):
            for p in range(3):
                for q in range(3):
                    T[a, b, p, q] = T[b, a, q, p] = float(integral(G[a][p] * G[b][q]))
    NI = np.array([float(integral(n)) for n in N])
    return T, NI


def test_pyr5_affine_pyramid_matches_exact_integration(oracle):
    """The 8-point collapsed rule integrates the stiffness of an affine pyramid
    exactly, so the oracle's element must equal the exact integral."""
    T, NI = _sym_ref_pyramid_tensors()
    assert NI.sum() == pytest.approx(4.0 / 3.0, rel=1e-15)
    rng = np.random.default_rng(17)
    A = np.eye(3) + rng.uniform(-0.3, 0.3, (3, 3))
    assert np.linalg.det(A) > 0
    X = np.array(REF_NODES[mg.PYR5], dtype=float) @ A.T + np.array([0.4, -1.2, 2.0])
    Ai = np.linalg.inv(A)
    P = np.linalg.det(A) * np.einsum("pk,ql,abpq->abkl", Ai, Ai, T)     # physical-gradient products
    Ae, be, _, _ = oracle.element(mg.PYR5, X, oracle.OP_DIFFUSION, k0=1.0, k2=0.0, source=1.5)
    exact = np.einsum("abkk->ab", P)
    assert np.allclose(Ae, exact, rtol=0, atol=1e-14 * np.abs(exact).max())
    assert np.allclose(be, 1.5 * np.linalg.det(A) * NI, rtol=1e-14, atol=0)
    E, nu = 2.1, 0.33
    lam = E * nu / ((1 + nu) * (1 - 2 * nu)); mu = E / (2 * (1 + nu))
    Ke, _, _, _ = oracle.element(mg.PYR5, X, oracle.OP_ELASTICITY, young=E, poisson=nu)
    K = np.zeros((15, 15))
    for a in range(5):
        for b in range(5):
            for c in range(3):
                for cc in range(3):
                    K[3 * a + c, 3 * b + cc] = (lam * P[a, b, c, cc] + mu * P[a, b, cc, c]
                                                + (mu * np.trace(P[a, b]) if c == cc else 0.0))
    assert np.allclose(Ke, K, rtol=0, atol=1e-13 * np.abs(K).max())


def test_tet4_variable_coefficient_closed_form(oracle):
    """k(x) = k0 + k2 x^2 at the physical x of the points: on a tet the
    gradients are constant, so A = (int k dV) G G^T.  The 4-point rule is
    exact for the quadratic k: int x^2 dV = V/20 (sum_a x_a^2 + (sum_a x_a)^2),
    from int lambda_a lambda_b dV = V (1 + delta_ab) / 20.  The 1-point rule
    takes k at the centroid."""
    rng = np.random.default_rng(23)
    X = np.array([[0.3, -0.2, 0.1], [1.4, 0.1, 0.0], [0.5, 1.2, 0.2], [0.6, 0.4, 1.3]]) + rng.uniform(-0.1, 0.1, (4, 3))
    E = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    V = np.linalg.det(E) / 6.0
    G = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float) @ np.linalg.inv(E)
    k0, k2 = 0.7, 2.3
    x = X[:, 0]
    int_k = k0 * V + k2 * V / 20.0 * (np.sum(x ** 2) + np.sum(x) ** 2)
    A4, _, _, _ = oracle.element(mg.TET4, X, oracle.OP_DIFFUSION, tet_rule=1, k0=k0, k2=k2)
    np.testing.assert_allclose(A4, int_k * G @ G.T, rtol=1e-13, atol=1e-15)
    A1, _, _, _ = oracle.element(mg.TET4, X, oracle.OP_DIFFUSION, tet_rule=0, k0=k0, k2=k2)
    np.testing.assert_allclose(A1, (k0 + k2 * x.mean() ** 2) * V * G @ G.T, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("rule", [0, 1])
def test_tet4_affine_closed_form(oracle, rule):
    rng = np.random.default_rng(5)
    X = np.array([[0, 0, 0], [1, 0.1, 0], [0.2, 1, 0.1], [0.1, 0.3, 1.2]]) + rng.uniform(-0.05, 0.05, (4, 3))
    E = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)   # columns = edges
    V = np.linalg.det(E) / 6.0
    Gref = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    G = Gref @ np.linalg.inv(E)
    Ae, be, _, _ = oracle.element(mg.TET4, X, oracle.OP_DIFFUSION, tet_rule=rule, k0=2.0, k2=0.0, source=3.0)
    assert np.allclose(Ae, 2.0 * V * G @ G.T, rtol=1e-13, atol=1e-15)
    assert np.allclose(be, 3.0 * V / 4.0, rtol=1e-13)
    D = _voigt_D(1.3, 0.2)
    B = np.zeros((6, 12))
    for a in range(4):
        gx, gy, gz = G[a]
        B[:, 3 * a:3 * a + 3] = [[gx, 0, 0], [0, gy, 0], [0, 0, gz], [gy, gx, 0], [0, gz, gy], [gz, 0, gx]]
    Ke, _, _, _ = oracle.element(mg.TET4, X, oracle.OP_ELASTICITY, tet_rule=rule, young=1.3, poisson=0.2)
    assert np.allclose(Ke, V * B.T @ D @ B, rtol=1e-12, atol=1e-14)


def test_pyramid_volume_and_rigid_modes(oracle):
    # pyramid over a square base of side 2 and height 1.5, apex off-centre
    X = np.array([(-1, -1, 0), (1, -1, 0), (1, 1, 0), (-1, 1, 0), (0.2, -0.1, 1.5)], dtype=float)
    Ae, be, _, _ = oracle.element(mg.PYR5, X, oracle.OP_DIFFUSION, source=1.0)
    assert abs(be.sum() - 4.0 * 1.5 / 3.0) < 1e-14
    assert np.allclose(Ae.sum(axis=1), 0.0, atol=1e-14)
    Ke, fe, _, _ = oracle.element(mg.PYR5, X, oracle.OP_ELASTICITY, body_force=(1, 1, 1))
    assert np.allclose(fe.reshape(5, 3).sum(axis=0), 2.0, rtol=1e-14)
    for r in _rigid_modes(X):
        assert np.abs(Ke @ r).max() < 1e-13 * np.abs(Ke).max()


def test_inverted_element_is_reported(oracle):
    m = mg.hex_cube(2)
    conn = m.conn.copy().reshape(-1, 8)
    conn[5] = conn[5][[4, 5, 6, 7, 0, 1, 2, 3]]       # mirror element 5 through its mid-plane
    m.conn = conn.reshape(-1)
    with pytest.raises(oracle.InvertedElement) as ei:
        oracle.assemble(m, oracle.OP_DIFFUSION)
    assert ei.value.elem == 5


# ----------------------------------------------------------------------------
# patterns
# ----------------------------------------------------------------------------

def _brute_pattern(mesh):
    n = mesh.n_nodes
    adj = np.zeros((n, n), dtype=bool)
    for e in range(mesh.n_elems):
        nodes = mesh.element_nodes(e)
        adj[np.ix_(nodes, nodes)] = True
    return adj


def _tiny_meshes():
    return [mg.kuhn_tet_cube(1), mg.hex_cube(2, 0.2, 7),
            mg.template_cube(1, mg.PYR5), mg.template_cube(2, mg.PRISM6),
            mg.template_cube(1, mg.HEX8), mg.hybrid_cube(2, 11)]


@pytest.mark.parametrize("idx", range(6))
@pytest.mark.parametrize("ndof", [1, 3])
def test_pattern_matches_brute_force(oracle, idx, ndof):
    mesh = _tiny_meshes()[idx]
    rp, col, nmap = oracle.pattern(mesh, ndof)
    adj = _brute_pattern(mesh)
    n = mesh.n_nodes
    for i in range(n):
        for c in range(ndof):
            row = col[rp[ndof * i + c]:rp[ndof * i + c + 1]]
            expect = (ndof * np.nonzero(adj[i])[0][:, None] + np.arange(ndof)[None, :]).ravel()
            assert np.array_equal(row, expect)
    # rank-map round trip: scalar entry (d*i+c, d*j+c') sits at rp[d*i+c] + d*k + c'
    off = 0
    for e in range(mesh.n_elems):
        nodes = mesh.element_nodes(e); ne = len(nodes)
        k = nmap[off:off + ne * ne].reshape(ne, ne)
        for a in range(ne):
            for b in range(ne):
                for c in range(ndof):
                    for cc in range(ndof):
                        assert col[rp[ndof * nodes[a] + c] + ndof * k[a, b] + cc] == ndof * nodes[b] + cc
        off += ne * ne


@pytest.mark.parametrize("n", [3, 6])
def test_pattern_closed_form_counts(oracle, n):
    rp, col, _ = oracle.pattern(mg.hex_cube(n), 1)
    assert len(col) == (3 * n + 1) ** 3                   # 27-point stencil, truncated at the faces
    assert np.diff(rp).max() == 27
    rp, col, _ = oracle.pattern(mg.hex_cube(n), 3)
    assert len(col) == 9 * (3 * n + 1) ** 3


def test_kuhn_pattern_nnz_closed_form(oracle):
    # 4913 diagonal + 2 x 31024 lattice edges (3 axis + 3 face-diagonal + 1 body-diagonal directions)
    n = 16
    edges = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    rp, col, _ = oracle.pattern(mg.kuhn_tet_cube(n), 1)
    assert len(col) == (n + 1) ** 3 + 2 * edges == 66961


# ----------------------------------------------------------------------------
# assembled systems
# ----------------------------------------------------------------------------

def _rows(rp):
    return np.repeat(np.arange(len(rp) - 1), np.diff(rp))


def _matvec(r, x):
    return np.bincount(_rows(r["row_ptr"]), weights=r["A"] * x[r["col_idx"]], minlength=len(r["row_ptr"]) - 1)


def _symmetric(r):
    """max |a_ij - a_ji| / S_ij (0 for a bit-symmetric matrix)."""
    import scipy.sparse as sps
    M = sps.csr_matrix((r["A"], r["col_idx"], r["row_ptr"]))
    S = sps.csr_matrix((r["SA"], r["col_idx"], r["row_ptr"]))
    D = abs(M - M.T).tocsr()
    D.sort_indices(); S.sort_indices()
    if D.nnz == 0:
        return 0.0
    Sd = S.multiply(D != 0).tocsr()
    return float(np.max(D.data / np.asarray(Sd[D.nonzero()]).ravel()))


def test_kuhn_poisson_pins(oracle):
    n = 16; h = 1.0 / n
    mesh = mg.kuhn_tet_cube(n)
    r = oracle.assemble(mesh, oracle.OP_DIFFUSION, tet_rule=0, k0=1.0, source=1.0)
    assert abs(r["b"].sum() - 1.0) < 1e-14
    rs = np.bincount(_rows(r["row_ptr"]), weights=r["A"])
    Srow = np.bincount(_rows(r["row_ptr"]), weights=r["SA"])
    assert np.all(np.abs(rs) <= 1e-14 * Srow)
    assert _symmetric(r) == 0.0
    # interior node: P1 on the Kuhn lattice is h times the 7-point stencil
    stride = {1: 1, 2: n + 1, 3: (n + 1) ** 2}
    for (i, j, k) in [(8, 8, 8), (1, 1, 1), (15, 3, 9)]:
        node = i + (n + 1) * (j + (n + 1) * k)
        cols = r["col_idx"][r["row_ptr"][node]:r["row_ptr"][node + 1]]
        vals = r["A"][r["row_ptr"][node]:r["row_ptr"][node + 1]]
        S = r["SA"][r["row_ptr"][node]:r["row_ptr"][node + 1]]
        assert len(cols) == 15
        for cj, v, s in zip(cols, vals, S):
            off = int(cj) - node
            if off == 0:
                assert abs(v - 6 * h) < 1e-15
            elif abs(off) in stride.values():
                assert abs(v + h) < 1e-16
            else:
                assert abs(v) <= 1e-15 * s
        assert abs(r["b"][node] - h ** 3) < 1e-18


@pytest.mark.parametrize("etype", [mg.TET4, mg.PRISM6, mg.HEX8])
def test_patch_test_on_distorted_meshes(oracle, etype):
    mesh = mg.hex_cube(4, 0.25, 3) if etype == mg.HEX8 else mg.template_cube(3, etype, 0.3, 4)
    x = mesh.coords
    interior = np.all((x > 1e-12) & (x < 1 - 1e-12), axis=1)
    rng = np.random.default_rng(9)
    # diffusion, k = 1: a linear field is in the kernel at interior nodes
    c = rng.normal(size=4)
    u = c[0] + x @ c[1:]
    r = oracle.assemble(mesh, oracle.OP_DIFFUSION, k0=1.0, k2=0.0)
    Au = _matvec(r, u)
    scale = np.bincount(_rows(r["row_ptr"]), weights=r["SA"] * np.abs(u[r["col_idx"]]))
    assert np.all(np.abs(Au[interior]) <= 1e-13 * scale[interior])
    assert np.abs(Au[~interior]).max() > 1e-6 * scale.max()      # non-trivial on the boundary
    # elasticity: a linear displacement field likewise
    M = rng.normal(size=(3, 3)); t = rng.normal(size=3)
    U = (x @ M.T + t).reshape(-1)
    r = oracle.assemble(mesh, oracle.OP_ELASTICITY)
    KU = _matvec(r, U).reshape(-1, 3)
    scale = np.bincount(_rows(r["row_ptr"]), weights=r["SA"] * np.abs(U[r["col_idx"]])).reshape(-1, 3)
    assert np.all(np.abs(KU[interior]) <= 1e-13 * scale[interior])


def _rigid_modes(x):
    modes = []
    for c in range(3):
        t = np.zeros_like(x); t[:, c] = 1.0
        modes.append(t.reshape(-1))
    for axis in range(3):
        w = np.zeros(3); w[axis] = 1.0
        modes.append(np.cross(w, x).reshape(-1))
    return modes


def test_elasticity_rigid_modes_symmetry_volume(oracle):
    mesh = mg.hex_cube(4, 0.2, 2)
    r = oracle.assemble(mesh, oracle.OP_ELASTICITY, young=1.0, poisson=0.3, body_force=(1, 1, 1))
    assert _symmetric(r) <= 1e-15
    for mode in _rigid_modes(mesh.coords):
        Kr = _matvec(r, mode)
        scale = np.bincount(_rows(r["row_ptr"]), weights=r["SA"] * np.abs(mode[r["col_idx"]]))
        assert np.all(np.abs(Kr) <= 1e-13 * scale + 1e-300)
    assert np.allclose(r["b"].reshape(-1, 3).sum(axis=0), 1.0, rtol=0, atol=1e-14)


def test_hybrid_mesh_invariants(oracle):
    mesh = mg.hybrid_cube(4, 3)
    r = oracle.assemble(mesh, oracle.OP_DIFFUSION, k0=1.0, k2=1.0, source=1.0)
    assert abs(r["b"].sum() - 1.0) < 1e-13
    rs = np.bincount(_rows(r["row_ptr"]), weights=r["A"])
    Srow = np.bincount(_rows(r["row_ptr"]), weights=r["SA"])
    assert np.all(np.abs(rs) <= 1e-14 * Srow)
    assert _symmetric(r) == 0.0
    assert np.all(r["SA"] >= np.abs(r["A"]))
    assert np.all(r["NA"] >= r["SA"] * (1 - 1e-14))          # Cauchy-Schwarz: normwise >= componentwise
    re = oracle.assemble(mesh, oracle.OP_ELASTICITY, young=1.0, poisson=0.3)
    assert np.all(re["NA"] >= re["SA"] * (1 - 1e-14))


def test_rows_function_equals_full_assembly(oracle):
    mesh = mg.hybrid_cube(3, 5)
    for op in (oracle.OP_DIFFUSION, oracle.OP_ELASTICITY):
        d = 1 if op == oracle.OP_DIFFUSION else 3
        full = oracle.assemble(mesh, op, k0=1.0, k2=1.0)
        nodes = [0, 7, mesh.n_nodes // 2, mesh.n_nodes - 1]
        rows = oracle.assemble_rows(mesh, nodes, op, k0=1.0, k2=1.0)
        for node, row in zip(nodes, rows):
            for c in range(d):
                s, e = full["row_ptr"][d * node + c], full["row_ptr"][d * node + c + 1]
                assert np.array_equal(full["A"][s:e], row["vals"][c])
                assert np.array_equal(full["SA"][s:e], row["svals"][c])
                assert full["b"][d * node + c] == row["b"][c]
