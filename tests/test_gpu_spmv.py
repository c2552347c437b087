"""GPU parity of the assembled-operator product and of its partial-row form
over an element partition (Sec. 3.1), against the oracle's global system."""
import numpy as np
import pytest

from paper_1805_03949_gb300 import meshgen as mg
from tests.helpers import engine

pytestmark = pytest.mark.gpu


def _global(oracle, mesh, kind, d):
    import scipy.sparse as sps
    r = oracle.assemble(mesh, kind, tet_rule=1, poisson=0.3, k0=1.0, k2=1.0)
    return sps.csr_matrix((r["A"], r["col_idx"], r["row_ptr"]), shape=(d * mesh.n_nodes, d * mesh.n_nodes))


@pytest.mark.parametrize("name", ["hex9", "hybrid4", "kuhn6", "ragged"])
@pytest.mark.parametrize("kind", [0, 1])
def test_spmv_matches_oracle_system(oracle, name, kind):
    import torch
    fea = engine()
    mesh = {"hex9": lambda: mg.hex_cube(9, 0.2, 2), "hybrid4": lambda: mg.hybrid_cube(4, 5),
            "kuhn6": lambda: mg.kuhn_tet_cube(6), "ragged": lambda: mg.hex_cube(0, 0.2, 5, nx=3, ny=1, nz=7)}[name]()
    d = 1 if kind == 0 else 3
    s = fea.System.from_mesh(mesh, d, with_cols=False)
    try:
        s.assemble(fea.make_operator(kind=kind, precision=0, tet_rule=1, poisson=0.3, k0=1.0, k2=1.0))
        x = np.random.default_rng(7).normal(size=d * mesh.n_nodes)
        y = torch.full((d * mesh.n_nodes,), float("nan"), dtype=torch.float64, device="cuda")
        fea.fea_spmv(s.handle, d, s.row_ptr, s.A, torch.tensor(x, device="cuda"), y)
        ref = _global(oracle, mesh, kind, d) @ x
        scale = np.abs(_global(oracle, mesh, kind, d)).max() * np.abs(x).max() * 30
        assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * scale
    finally:
        s.close()


@pytest.mark.parametrize("parts", [2, 5])
@pytest.mark.parametrize("precision", [0, 1])
def test_partial_row_product_over_a_partition(oracle, parts, precision):
    """Each subdomain assembles its own square local matrix on the GPU; the
    products of the subdomains, summed at interface nodes, equal the global
    system's product."""
    import torch
    fea = engine()
    mesh = mg.hybrid_cube(5, 4)
    d = 3
    subs, mult = mg.partition_elements(mesh, parts)
    x = np.random.default_rng(3).normal(size=d * mesh.n_nodes)
    xd = torch.tensor(x, device="cuda")
    y = torch.zeros(d * mesh.n_nodes, dtype=torch.float64, device="cuda")
    systems = []
    try:
        for sub, glob in subs:
            s = fea.System.from_mesh(sub, d, with_cols=False)
            systems.append(s)
            s.assemble(fea.make_operator(kind=1, precision=precision, tet_rule=1, poisson=0.3))
            g = torch.tensor(glob, device="cuda")
            sh = torch.tensor((mult[glob] > 1).astype(np.uint8), device="cuda")
            fea.fea_spmv(s.handle, d, s.row_ptr, s.A, xd, y, g, sh)
        A = _global(oracle, mesh, 1, d)
        ref = A @ x
        scale = np.abs(A).max() * np.abs(x).max() * 30
        tol = 1e-12 if precision == 0 else 1e-5
        assert np.abs(y.cpu().numpy() - ref).max() <= tol * scale
    finally:
        for s in systems:
            s.close()
