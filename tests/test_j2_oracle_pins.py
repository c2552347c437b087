"""Pins of the J2 / Voce oracle (CPU only) against closed forms, an independent
solver and finite differences -- never against the oracle itself.

The material model is small-strain J2 plasticity with isotropic Voce
hardening, integrated by the radial return map with its consistent tangent
(the constitutive update at the Gauss points of the solid mechanics element
loop, Sec. 2.2 / 5.2 of the paper).
"""
import numpy as np
import pytest

from paper_1805_03949_gb300 import meshgen as mg

E, NU = 1.0, 0.3
LAM = E * NU / ((1 + NU) * (1 - 2 * NU))
MU = E / (2 * (1 + NU))


def _voigt_elastic():
    """Textbook isotropic D on engineering strain (Voigt xx, yy, zz, xy, yz, xz)."""
    D = np.zeros((6, 6))
    D[:3, :3] = LAM
    D[np.arange(3), np.arange(3)] = LAM + 2 * MU
    D[np.arange(3, 6), np.arange(3, 6)] = MU
    return D


def _eng(eps):
    """Tensor components -> engineering strain vector."""
    e = np.array(eps, dtype=float)
    return np.concatenate([e[:3], 2 * e[3:]])


def _dev_norm(s):
    m = np.array(s[:3]).mean()
    d = np.array(s, dtype=float) - np.array([m, m, m, 0, 0, 0])
    return np.sqrt((d[:3] ** 2).sum() + 2 * (d[3:] ** 2).sum())


def _voce(a, s0=1e-3, sinf=3e-3, delta=300.0, H=1e-2):
    return s0 + H * a + (sinf - s0) * (1 - np.exp(-delta * a))


STRAINS = [
    [2e-3, -1e-3, 5e-4, 1e-3, -2e-3, 3e-4],
    [1e-2, 0, 0, 0, 0, 0],
    [0, 0, 0, 4e-3, 0, 0],
    [3e-3, 3e-3, -6e-3, 0, 1e-3, 0],
    [5e-2, -2e-2, 1e-2, 3e-2, 0, -1e-2],
]


def test_elastic_point_gives_textbook_stiffness(oracle):
    eps = np.array([1e-5, -2e-5, 3e-6, 4e-6, -1e-6, 2e-6])
    r = oracle.j2_point(eps)
    assert r["yielded"] == 0 and r["iters"] == 0
    D = _voigt_elastic()
    np.testing.assert_allclose(r["D"], D, rtol=0, atol=1e-15)
    np.testing.assert_allclose(r["sigma"], D @ _eng(eps), rtol=1e-14, atol=1e-20)
    np.testing.assert_array_equal(r["eps_p"], 0.0)


def test_linear_hardening_closed_form(oracle):
    """sigma_inf = sigma0: the consistency condition is linear, dg = f / (2 mu + 2/3 H)."""
    H = 0.05
    for eps in STRAINS:
        r = oracle.j2_point(eps, sigma0=1e-3, sigma_inf=1e-3, hardening=H)
        e = np.array(eps, dtype=float)
        tr = e[:3].sum()
        s = 2 * MU * (e - np.array([tr / 3] * 3 + [0] * 3))
        norm = np.sqrt((s[:3] ** 2).sum() + 2 * (s[3:] ** 2).sum())
        f = norm - np.sqrt(2 / 3) * 1e-3
        assert f > 0 and r["yielded"] == 1
        dg = f / (2 * MU + 2 / 3 * H)
        assert r["alpha"] == pytest.approx(np.sqrt(2 / 3) * dg, rel=1e-13)
        assert r["iters"] == 1                       # one Newton step solves a linear condition
        np.testing.assert_allclose(r["eps_p"], dg * s / norm, rtol=1e-12, atol=1e-18)


def _bisect_dg(eps, alpha_n=0.0, eps_p_n=None):
    """Root of the consistency condition by bisection (independent of the oracle's Newton)."""
    e = np.array(eps, dtype=float) - (0 if eps_p_n is None else np.asarray(eps_p_n))
    tr = e[:3].sum()
    s = 2 * MU * (e - np.array([tr / 3] * 3 + [0] * 3))
    norm = np.sqrt((s[:3] ** 2).sum() + 2 * (s[3:] ** 2).sum())
    g = lambda dg: norm - 2 * MU * dg - np.sqrt(2 / 3) * _voce(alpha_n + np.sqrt(2 / 3) * dg)
    lo, hi = 0.0, norm / (2 * MU)
    assert g(lo) > 0 > g(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("k", range(len(STRAINS)))
def test_voce_return_map_matches_bisection_and_yield_surface(oracle, k):
    eps = STRAINS[k]
    r = oracle.j2_point(eps)
    assert r["yielded"] == 1 and 1 <= r["iters"] <= 12
    dg = _bisect_dg(eps)
    assert r["alpha"] == pytest.approx(np.sqrt(2 / 3) * dg, rel=1e-11)
    # the returned stress lies on the updated yield surface
    assert _dev_norm(r["sigma"]) == pytest.approx(np.sqrt(2 / 3) * _voce(r["alpha"]), rel=1e-11)
    # plastic flow is deviatoric and along the trial direction
    assert abs(r["eps_p"][:3].sum()) <= 1e-15
    assert abs(np.sqrt((r["eps_p"][:3] ** 2).sum() + 2 * (r["eps_p"][3:] ** 2).sum()) - dg) <= 1e-12 * dg


def test_return_map_with_prior_state(oracle):
    """A second load step from a committed state: same bisection pin with alpha_n, eps_p_n."""
    r1 = oracle.j2_point(STRAINS[0])
    eps2 = np.array(STRAINS[0]) * 1.7
    r2 = oracle.j2_point(eps2, r1["eps_p"], r1["alpha"])
    dg = _bisect_dg(eps2, r1["alpha"], r1["eps_p"])
    assert r2["alpha"] - r1["alpha"] == pytest.approx(np.sqrt(2 / 3) * dg, rel=1e-10)
    # reloading to the committed strain from the committed state is (to rounding) elastic
    r3 = oracle.j2_point(STRAINS[0], r1["eps_p"], r1["alpha"])
    assert r3["alpha"] - r1["alpha"] <= 1e-13 * r1["alpha"]


@pytest.mark.parametrize("k", range(len(STRAINS)))
def test_consistent_tangent_matches_finite_differences(oracle, k):
    eps = np.array(STRAINS[k], dtype=float)
    epn = np.array([1e-4, -5e-5, -5e-5, 2e-5, 0, 1e-5]) if k % 2 else np.zeros(6)
    an = 1e-3 if k % 2 else 0.0
    r = oracle.j2_point(eps, epn, an)
    h = 1e-7 * max(1e-3, np.abs(eps).max())
    Dfd = np.zeros((6, 6))
    for j in range(6):
        d = np.zeros(6)
        d[j] = h if j < 3 else h / 2                 # engineering shear perturbation h
        sp = oracle.j2_point(eps + d, epn, an)["sigma"]
        sm = oracle.j2_point(eps - d, epn, an)["sigma"]
        Dfd[:, j] = (sp - sm) / (2 * h)
    scale = np.abs(r["D"]).max()
    assert np.abs(r["D"] - Dfd).max() <= 1e-6 * scale
    np.testing.assert_allclose(r["D"], r["D"].T, rtol=0, atol=1e-14 * scale)   # associative flow


def test_max_iter_failure_is_reported(oracle):
    with pytest.raises(oracle.NoConvergence):
        oracle.j2_point(STRAINS[4], max_iter=1, tol_step=0.0)


def _hex_element(jitter_seed=3):
    m = mg.hex_cube(1, 0.0)
    X = m.coords[m.conn[:8]].copy()
    X += np.random.default_rng(jitter_seed).uniform(-0.1, 0.1, X.shape)
    return X


def _rigid_modes(X):
    modes = []
    for c in range(3):
        t = np.zeros_like(X); t[:, c] = 1.0
        modes.append(t.reshape(-1))
    for axis in range(3):
        w = np.zeros(3); w[axis] = 1.0
        modes.append(np.cross(w, X).reshape(-1))
    return modes


NODES = {mg.TET4: 4, mg.PYR5: 5, mg.PRISM6: 6, mg.HEX8: 8}
ALL_TYPES = [mg.HEX8, mg.TET4, mg.PYR5, mg.PRISM6]


def _element(etype):
    if etype == mg.HEX8:
        return _hex_element()
    m = mg.template_cube(1, etype, 0.0)
    return m.coords[m.conn[:NODES[etype]]].copy()


@pytest.mark.parametrize("etype", ALL_TYPES)
def test_element_invariants(oracle, etype):
    X = _element(etype)
    nn = X.shape[0]
    U = 4e-3 * np.sin(3.0 * X + np.array([0.3, 1.1, 2.0]))
    r = oracle.j2_element(etype, X, U)
    assert r["yielded"].sum() > 0                     # the load reaches the plastic range
    A, f = r["A"], r["b"]
    scale = np.abs(A).max()
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-13 * scale)
    # sum over nodes of the internal force vanishes (sum_a grad N_a = 0)
    assert np.abs(f.reshape(nn, 3).sum(axis=0)).max() <= 1e-14 * np.abs(f).max()
    for mode in _rigid_modes(X):
        assert np.abs(A @ mode).max() <= 1e-13 * scale * np.abs(mode).max()


@pytest.mark.parametrize("etype", ALL_TYPES)
def test_elastic_element_equals_linear_elasticity(oracle, etype):
    """Below yield: tangent = the linear elastic element matrix, f_int = K u."""
    X = _element(etype)
    U = 1e-6 * np.cos(2.0 * X)
    r = oracle.j2_element(etype, X, U)
    assert r["yielded"].sum() == 0
    K, _, _, _ = oracle.element(etype, X, oracle.OP_ELASTICITY, young=E, poisson=NU, body_force=(0, 0, 0),
                                tet_rule=1)
    np.testing.assert_allclose(r["A"], K, rtol=0, atol=1e-14 * np.abs(K).max())
    np.testing.assert_allclose(r["b"], K @ U.reshape(-1), rtol=0, atol=1e-13 * np.abs(K).max() * 1e-6)


@pytest.mark.parametrize("etype", ALL_TYPES)
def test_element_tangent_is_the_force_derivative(oracle, etype):
    """In the plastic range the element matrix is the derivative of the
    internal force with respect to the nodal displacements (the committed
    state fixed): central differences, no point changing between elastic and
    plastic under the perturbation."""
    X = _element(etype) + np.random.default_rng(3).uniform(-0.05, 0.05, (NODES[etype], 3))
    U = 4e-3 * np.sin(3.0 * X + np.array([0.3, 1.1, 2.0]))
    r = oracle.j2_element(etype, X, U)
    assert r["yielded"].sum() > 0
    n, h = U.size, 1e-9
    Kfd = np.zeros((n, n))
    for j in range(n):
        d = np.zeros(n); d[j] = h
        rp = oracle.j2_element(etype, X, (U.reshape(-1) + d).reshape(U.shape))
        rm = oracle.j2_element(etype, X, (U.reshape(-1) - d).reshape(U.shape))
        assert (rp["yielded"] == r["yielded"]).all() and (rm["yielded"] == r["yielded"]).all()
        Kfd[:, j] = (rp["b"] - rm["b"]) / (2 * h)
    np.testing.assert_allclose(r["A"], Kfd, rtol=0, atol=1e-7 * np.abs(r["A"]).max())


def test_global_assembly_invariants(oracle):
    mesh = mg.hex_cube(4, 0.2, 4)
    U = mg.fourier_displacement(mesh.coords, 2e-4, seed=4)
    r1 = oracle.j2_assemble(mesh, 0.5 * U)
    r2 = oracle.j2_assemble(mesh, U, r1["state"])
    assert 0 < r2["yielded"].mean() < 1
    assert (r2["yielded"] >= r1["yielded"]).all()     # proportional loading: yielded points keep yielding
    import scipy.sparse as sps
    K = sps.csr_matrix((r2["A"], r2["col_idx"], r2["row_ptr"]))
    scale = abs(K).max()
    assert abs(K - K.T).max() <= 1e-13 * scale
    for mode in _rigid_modes(mesh.coords):
        assert np.abs(K @ mode).max() <= 1e-12 * scale
    f = r2["b"].reshape(-1, 3)
    assert np.abs(f.sum(axis=0)).max() <= 1e-13 * np.abs(f).max() * mesh.n_nodes ** 0.5
    assert r2["iters"].max() <= 12
    # the point sweep counts the same yielded points as the assembly
    n1, st1 = oracle.j2_sweep(mesh, U, 0.5, want_state=True)
    assert n1 == int(r1["yielded"].sum())
    np.testing.assert_array_equal(st1, r1["state"])
    assert oracle.j2_sweep(mesh, U, 1.0, st1) == int(r2["yielded"].sum())


def test_point_loop_agrees_with_the_assembly_and_its_stress_gives_f_int(oracle):
    """The element-wise loop's state, flags and counts equal the assembly's; its
    stresses, pushed through B^T by numpy, rebuild the internal force vector."""
    mesh = mg.hex_cube(3, 0.2, 4)
    U = mg.fourier_displacement(mesh.coords, 1.5e-4, seed=4)
    r1 = oracle.j2_assemble(mesh, 0.5 * U)
    r2 = oracle.j2_assemble(mesh, U, r1["state"])
    pts = oracle.j2_points(mesh, U, r1["state"])
    np.testing.assert_array_equal(pts["state"], r2["state"])
    np.testing.assert_array_equal(pts["iters"], r2["iters"])
    np.testing.assert_array_equal(pts["yielded"], r2["yielded"])
    assert 0 < pts["n_yielded"] < 8 * mesh.n_elems
    q, w = oracle.quadrature(mg.HEX8)
    f = np.zeros((mesh.n_nodes, 3))
    for e in range(mesh.n_elems):
        nodes = mesh.element_nodes(e)
        X = mesh.coords[nodes]
        for k in range(8):
            _, dN = oracle.shape(mg.HEX8, q[k])
            J = X.T @ dN
            G = dN @ np.linalg.inv(J)
            s = pts["stress"][e, k]
            S = np.array([[s[0], s[3], s[5]], [s[3], s[1], s[4]], [s[5], s[4], s[2]]])
            f[nodes] += w[k] * np.linalg.det(J) * G @ S
    np.testing.assert_allclose(f.reshape(-1), r2["b"], rtol=0, atol=1e-12 * np.abs(r2["b"]).max())
