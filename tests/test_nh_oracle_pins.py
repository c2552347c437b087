"""Pins of the finite-strain (neo-Hookean, first Piola-Kirchhoff) oracle, CPU
only: the linear-elastic limit, derivatives by central finite differences
(stress of the energy, tangent of the stress, element Jacobian of the
internal force, internal force of the stored energy), frame indifference,
the balance of angular momentum, a finite rigid rotation, the traction of a
homogeneous stretch and the mass integral -- never the oracle against itself.

The reading (Sec. 2.2 of the paper names no material): the compressible
neo-Hookean solid of Bonet and Wood, with the Newmark mass term in the
Jacobian.
"""
import numpy as np
import pytest

from paper_1805_03949_gb300 import meshgen as mg

E, NU = 1.0, 0.3
LAM = E * NU / ((1 + NU) * (1 - 2 * NU))
MU = E / (2 * (1 + NU))
EYE = np.eye(3)


def _rot(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    return q if np.linalg.det(q) > 0 else -q


def _F(seed, amp=0.3):
    return EYE + amp * np.random.default_rng(seed).uniform(-1, 1, (3, 3))


def _elements():
    out = {}
    m = mg.hex_cube(1, 0.0)
    X = m.coords[m.conn[:8]].copy()
    X += np.random.default_rng(3).uniform(-0.1, 0.1, X.shape)
    out[mg.HEX8] = X
    for t in (mg.TET4, mg.PYR5, mg.PRISM6):
        m = mg.template_cube(1, t, 0.0)
        out[t] = m.coords[m.conn[:int(m.conn_offsets[1])]].copy()
    return out


ELEMS = _elements()


def _U(X, amp=0.08, seed=5):
    """A smooth finite deformation (strains of a few 10 %)."""
    ph = np.random.default_rng(seed).uniform(0, 2 * np.pi, 3)
    return amp * np.sin(2.5 * X + ph) + 0.1 * amp * X[:, [1, 2, 0]]


def test_reference_state_gives_the_linear_elastic_tensor(oracle):
    r = oracle.nh_point(EYE)
    assert r["psi"] == 0.0 and np.abs(r["P"]).max() == 0.0
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[i, j, k, l] = LAM * (i == j) * (k == l) + MU * ((i == k) * (j == l) + (i == l) * (j == k))
    np.testing.assert_allclose(r["A"], C, rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_stress_is_the_energy_derivative(oracle, seed):
    F = _F(seed)
    r = oracle.nh_point(F)
    h = 1e-6
    P = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            d = np.zeros((3, 3)); d[i, j] = h
            P[i, j] = (oracle.nh_point(F + d)["psi"] - oracle.nh_point(F - d)["psi"]) / (2 * h)
    np.testing.assert_allclose(r["P"], P, rtol=0, atol=1e-8 * np.abs(P).max())


@pytest.mark.parametrize("seed", range(4))
def test_tangent_is_the_stress_derivative(oracle, seed):
    F = _F(seed + 10)
    r = oracle.nh_point(F)
    h = 1e-6
    A = np.zeros((3, 3, 3, 3))
    for k in range(3):
        for l in range(3):
            d = np.zeros((3, 3)); d[k, l] = h
            A[:, :, k, l] = (oracle.nh_point(F + d)["P"] - oracle.nh_point(F - d)["P"]) / (2 * h)
    np.testing.assert_allclose(r["A"], A, rtol=0, atol=1e-8 * np.abs(A).max())


@pytest.mark.parametrize("seed", range(3))
def test_frame_indifference_and_angular_momentum(oracle, seed):
    F = _F(seed + 20)
    Q = _rot(seed)
    r, rq = oracle.nh_point(F), oracle.nh_point(Q @ F)
    assert rq["psi"] == pytest.approx(r["psi"], rel=1e-13)
    np.testing.assert_allclose(rq["P"], Q @ r["P"], rtol=0, atol=1e-14 * np.abs(r["P"]).max())
    tau = r["P"] @ F.T                                   # Kirchhoff stress is symmetric
    np.testing.assert_allclose(tau, tau.T, rtol=0, atol=1e-14 * np.abs(tau).max())


def test_small_strain_limit_is_linear_elasticity(oracle):
    H = np.random.default_rng(7).uniform(-1, 1, (3, 3))
    errs = []
    for eps in (1e-3, 1e-4):
        e = 0.5 * eps * (H + H.T)
        sig = LAM * np.trace(e) * EYE + 2 * MU * e
        errs.append(np.abs(oracle.nh_point(EYE + eps * H)["P"] - sig).max())
    assert errs[0] <= 10 * 1e-6 and errs[1] <= errs[0] / 50      # O(eps^2)


def test_inverted_deformation_is_rejected(oracle):
    with pytest.raises(oracle.InvertedElement):
        oracle.nh_point(np.diag([1.0, 1.0, -0.5]))


@pytest.mark.parametrize("etype", [mg.TET4, mg.PYR5, mg.PRISM6, mg.HEX8])
def test_element_at_rest_is_the_linear_elastic_element(oracle, etype):
    X = ELEMS[etype]
    r = oracle.nh_element(etype, X, np.zeros_like(X))
    K, _, _, _ = oracle.element(etype, X, oracle.OP_ELASTICITY, young=E, poisson=NU, body_force=(0, 0, 0))
    np.testing.assert_allclose(r["A"], K, rtol=0, atol=1e-14 * np.abs(K).max())
    assert np.abs(r["b"]).max() == 0.0 and r["energy"] == 0.0


@pytest.mark.parametrize("etype", [mg.TET4, mg.PYR5, mg.PRISM6, mg.HEX8])
def test_element_jacobian_is_the_force_derivative(oracle, etype):
    X = ELEMS[etype]
    U = _U(X)
    r = oracle.nh_element(etype, X, U)
    n = U.size
    h = 1e-6
    Kfd = np.zeros((n, n))
    for j in range(n):
        d = np.zeros(n); d[j] = h
        bp = oracle.nh_element(etype, X, (U.reshape(-1) + d).reshape(U.shape))["b"]
        bm = oracle.nh_element(etype, X, (U.reshape(-1) - d).reshape(U.shape))["b"]
        Kfd[:, j] = (bp - bm) / (2 * h)
    scale = np.abs(r["A"]).max()
    np.testing.assert_allclose(r["A"], Kfd, rtol=0, atol=1e-7 * scale)
    np.testing.assert_allclose(r["A"], r["A"].T, rtol=0, atol=1e-13 * scale)   # hyperelastic: symmetric


@pytest.mark.parametrize("etype", [mg.TET4, mg.PYR5, mg.PRISM6, mg.HEX8])
def test_element_force_is_the_energy_derivative(oracle, etype):
    X = ELEMS[etype]
    U = _U(X, seed=9)
    r = oracle.nh_element(etype, X, U)
    n = U.size
    h = 1e-6
    g = np.zeros(n)
    for j in range(n):
        d = np.zeros(n); d[j] = h
        ep = oracle.nh_element(etype, X, (U.reshape(-1) + d).reshape(U.shape))["energy"]
        em = oracle.nh_element(etype, X, (U.reshape(-1) - d).reshape(U.shape))["energy"]
        g[j] = (ep - em) / (2 * h)
    np.testing.assert_allclose(r["b"], g, rtol=0, atol=1e-8 * np.abs(g).max())


@pytest.mark.parametrize("etype", [mg.TET4, mg.PYR5, mg.PRISM6, mg.HEX8])
def test_finite_rigid_rotation_is_stress_free_and_rotates_the_jacobian(oracle, etype):
    X = ELEMS[etype]
    U = _U(X, seed=11)
    Q = _rot(42)                                         # a large rotation, not an infinitesimal one
    r0 = oracle.nh_element(etype, X, U)
    rr = oracle.nh_element(etype, X, X @ Q.T - X)        # x = Q X: F = Q everywhere
    assert np.abs(rr["b"]).max() <= 1e-14 and abs(rr["energy"]) <= 1e-14
    rq = oracle.nh_element(etype, X, (X + U) @ Q.T - X)  # the deformed shape, rotated
    nn = X.shape[0]
    fb = r0["b"].reshape(nn, 3)
    np.testing.assert_allclose(rq["b"].reshape(nn, 3), fb @ Q.T, rtol=0, atol=1e-13 * np.abs(fb).max())
    A0 = r0["A"].reshape(nn, 3, nn, 3)
    Aq = rq["A"].reshape(nn, 3, nn, 3)
    want = np.einsum("ij,ajbk,lk->aibl", Q, A0, Q)
    np.testing.assert_allclose(Aq, want, rtol=0, atol=1e-13 * np.abs(A0).max())
    assert rq["energy"] == pytest.approx(r0["energy"], rel=1e-12)


def test_homogeneous_stretch_gives_the_face_traction(oracle):
    """u = (F - I) X on a jittered unit cube: F is exact at every point, the
    interior forces vanish and the nodal forces on the face x = 1 add up to
    the traction P e_x times the face area 1."""
    mesh = mg.hex_cube(3, 0.2, 6)
    F = np.array([[1.3, 0.1, 0.0], [0.05, 0.9, 0.02], [0.0, -0.04, 1.1]])
    U = mesh.coords @ (F - EYE).T
    r = oracle.nh_assemble(mesh, U)
    f = r["b"].reshape(-1, 3)
    X = mesh.coords
    on_face = np.isclose(X[:, 0], 1.0)
    boundary = np.any(np.isclose(X, 0.0) | np.isclose(X, 1.0), axis=1)
    P = oracle.nh_point(F)["P"]
    np.testing.assert_allclose(f[on_face].sum(axis=0), P[:, 0], rtol=1e-12, atol=1e-14)
    assert np.abs(f[~boundary]).max() <= 1e-13 * np.abs(P).max()
    assert np.abs(f.sum(axis=0)).max() <= 1e-13 * np.abs(P).max()


def test_mass_term_integrates_the_volume(oracle):
    mesh = mg.hybrid_cube(3, 5)
    U = mg.fourier_displacement(mesh.coords, 0.01, seed=2)
    r0 = oracle.nh_assemble(mesh, U)
    r1 = oracle.nh_assemble(mesh, U, mass=2.5)
    assert (r1["A"] - r0["A"]).sum() == pytest.approx(3 * 2.5 * 1.0, rel=1e-12)   # 3 components x m x volume
    np.testing.assert_array_equal(r1["b"], r0["b"])
