"""GPU parity of the finite-strain solid (Sec. 2.2: first Piola-Kirchhoff
stress, Newton Jacobian with the Newmark mass term; compressible neo-Hookean
reading) against the oracle, on every element type, both precisions and
both scatters, plus the error paths."""
import numpy as np
import pytest

from paper_1805_03949_gb300 import meshgen as mg
from tests.helpers import FP32_TOL, FP64_TOL, engine, err_vs_oracle

pytestmark = pytest.mark.gpu

_MESHES = {
    "hex9": lambda: mg.hex_cube(9, 0.2, 2),
    "hybrid4": lambda: mg.hybrid_cube(4, 5),
    "kuhn5": lambda: mg.kuhn_tet_cube(5),
    "ragged": lambda: mg.hex_cube(0, 0.2, 5, nx=3, ny=1, nz=7),
}
_REF = {}


def _U(mesh, amp=0.004):
    """A smooth deformation with strains of several per cent."""
    return mg.fourier_displacement(mesh.coords, amp, seed=6) + 0.05 * mesh.coords[:, [1, 2, 0]]


def _ref(oracle, name, mesh, U, mass):
    key = (name, mass)
    if key not in _REF:
        _REF[key] = oracle.nh_assemble(mesh, U, young=1.0, poisson=0.3, mass=mass)
    return _REF[key]


@pytest.mark.parametrize("name", list(_MESHES))
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scatter", [0, 1])
@pytest.mark.parametrize("mass", [0.0, 2.0])
def test_neohooke_matches_oracle(oracle, name, precision, scatter, mass):
    import torch
    fea = engine()
    mesh = _MESHES[name]()
    U = _U(mesh)
    ref = _ref(oracle, name, mesh, U, mass)
    s = fea.System.from_mesh(mesh, 3)
    try:
        u = torch.tensor(U.reshape(-1), device="cuda")
        s.A.fill_(float("nan")); s.b.fill_(float("nan"))
        s.assemble(fea.make_operator(kind=fea.FEA_OP_NEOHOOKE, precision=precision, scatter=scatter, u=u,
                                     young=1.0, poisson=0.3, mass=mass))
        s.check()
        tol = FP64_TOL if precision == 0 else FP32_TOL
        errA, zA = err_vs_oracle(s.A.cpu().numpy(), ref["A"], ref["NA"])
        errb, zb = err_vs_oracle(s.b.cpu().numpy(), ref["b"], ref["Nb"])
        assert max(errA, errb, zA, zb) <= tol, (errA, errb, zA, zb)
        # the deformation is a finite one: the Jacobian differs from the linear one
        lin = oracle.nh_assemble(mesh, np.zeros_like(U), mass=mass)["A"]
        assert np.abs(ref["A"] - lin).max() > 1e3 * tol * np.abs(lin).max()
    finally:
        s.close()


def test_inverted_deformation_is_reported():
    import torch
    fea = engine()
    mesh = mg.hex_cube(3)
    U = np.zeros_like(mesh.coords)
    inner = np.nonzero(np.all((mesh.coords > 0.1) & (mesh.coords < 0.9), axis=1))[0][0]
    U[inner, 0] = 2.0                                   # drags one node through its elements
    s = fea.System.from_mesh(mesh, 3)
    try:
        u = torch.tensor(U.reshape(-1), device="cuda")
        s.assemble(fea.make_operator(kind=fea.FEA_OP_NEOHOOKE, precision=1, u=u))
        with pytest.raises(fea.FeaError) as e:
            s.check()
        assert e.value.code == -4
    finally:
        s.close()


def test_unsupported_and_invalid_requests_fail_on_the_host():
    import torch
    fea = engine()
    mesh = mg.hex_cube(2)
    s = fea.System.from_mesh(mesh, 3)
    try:
        u = torch.zeros(3 * mesh.n_nodes, dtype=torch.float64, device="cuda")
        with pytest.raises(fea.FeaError) as e:
            s.assemble(fea.make_operator(kind=fea.FEA_OP_NEOHOOKE, u=None))
        assert e.value.code == -1
        with pytest.raises(fea.FeaError) as e:
            s.assemble(fea.make_operator(kind=fea.FEA_OP_NEOHOOKE, u=u, schedule=fea.FEA_SCHED_STEAL))
        assert e.value.code == -8
        with pytest.raises(fea.FeaError) as e:
            s.assemble(fea.make_operator(kind=fea.FEA_OP_NEOHOOKE, u=u, scatter=fea.FEA_SCATTER_ROWS))
        assert e.value.code == -8
        with pytest.raises(fea.FeaError) as e:
            s.assemble(fea.make_operator(kind=fea.FEA_OP_NEOHOOKE, u=u, mass=-1.0))
        assert e.value.code == -1
    finally:
        s.close()
