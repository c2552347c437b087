"""GPU parity: CUDA pattern/map bit-exact and assembled values within tolerance of the oracle.

Every comparison goes through the C-ABI (via the thin binding) on seeded meshes
from ``meshgen``; the expected values come from the CPU oracle only.
"""
import numpy as np
import pytest

from paper_1805_03949_gb300 import meshgen as mg
from tests.helpers import FP32_TOL, FP64_TOL, engine, err_vs_oracle

pytestmark = pytest.mark.gpu


def _meshes_small():
    return {
        "kuhn1": lambda: mg.kuhn_tet_cube(1),
        "hex2j": lambda: mg.hex_cube(2, 0.2, 7),
        "pyr1": lambda: mg.template_cube(1, mg.PYR5),
        "prism2": lambda: mg.template_cube(2, mg.PRISM6, 0.2, 3),
        "hexref1": lambda: mg.template_cube(1, mg.HEX8),
        "hybrid2": lambda: mg.hybrid_cube(2, 11),
        "kuhn16": lambda: mg.kuhn_tet_cube(16),
        "hex12j": lambda: mg.hex_cube(12, 0.2, 2),
        "hybrid8": lambda: mg.hybrid_cube(8, 3),
        "ragged_hex": lambda: mg.hex_cube(0, 0.2, 5, nx=3, ny=4, nz=5),
        "one_tet": lambda: mg.kuhn_tet_cube(0, 1, 1, 1),
    }


@pytest.mark.parametrize("name", list(_meshes_small()))
@pytest.mark.parametrize("ndof", [1, 3])
def test_pattern_and_map_bit_exact(oracle, name, ndof):
    fea = engine()
    mesh = _meshes_small()[name]()
    if name == "one_tet":
        mesh.types = mesh.types[:1]; mesh.conn_offsets = mesh.conn_offsets[:2]; mesh.conn = mesh.conn[:4]
    s = fea.System.from_mesh(mesh, ndof)
    try:
        rp, col, nmap = oracle.pattern(mesh, ndof)
        assert np.array_equal(s.row_ptr.cpu().numpy(), rp)
        assert np.array_equal(s.col_idx.cpu().numpy(), col)
        assert np.array_equal(s.node_map.cpu().numpy(), nmap)
    finally:
        s.close()


CASES = {
    # name: (mesh factory, op kind, oracle op, tet_rule, params)
    "kuhn16_poisson": (lambda: mg.kuhn_tet_cube(16), 0, 0, 0, dict(k0=1.0, k2=0.0, source=1.0)),
    "hex10_elasticity": (lambda: mg.hex_cube(10, 0.2, 2), 1, 1, 1, dict(young=1.0, poisson=0.3)),
    "hex10_diffusion": (lambda: mg.hex_cube(10, 0.2, 2), 0, 0, 1, dict(k0=1.0, k2=1.0, source=1.0)),
    "hybrid6_diffusion": (lambda: mg.hybrid_cube(6, 3), 0, 0, 1, dict(k0=1.0, k2=1.0, source=1.0)),
    "hybrid5_elasticity": (lambda: mg.hybrid_cube(5, 4), 1, 1, 1, dict(young=2.0, poisson=0.25)),
    "pyr3_elasticity": (lambda: mg.template_cube(3, mg.PYR5, 0.2, 8), 1, 1, 1, dict(young=1.0, poisson=0.3)),
    "prism3_elasticity": (lambda: mg.template_cube(3, mg.PRISM6, 0.2, 8), 1, 1, 1, dict(young=1.0, poisson=0.3)),
    "tet3_elasticity_4pt": (lambda: mg.template_cube(3, mg.TET4, 0.2, 8), 1, 1, 1, dict(young=1.0, poisson=0.3)),
    "ragged_hex_elasticity": (lambda: mg.hex_cube(0, 0.2, 5, nx=3, ny=4, nz=5), 1, 1, 1, dict(poisson=0.3)),
    "stretched_hex_elasticity": (lambda: mg.hex_cube(0, 0.1, 6, nx=2, ny=3, nz=40), 1, 1, 1, dict(poisson=0.3)),
}


SCATTERS = {"atomic": 0, "color": 1, "block": 2, "rows": 3}


_ORACLE_CACHE = {}


def _reference(oracle, name, mesh):
    """Oracle system of a case (computed once per case; every precision and scatter compares to it)."""
    if name not in _ORACLE_CACHE:
        _, _, oop, tet_rule, params = CASES[name]
        _ORACLE_CACHE[name] = oracle.assemble(mesh, oop, tet_rule=tet_rule, **params)
    return _ORACLE_CACHE[name]


def _run_case(fea, oracle, name, precision, scatter=0, block_nodes=None):
    factory, kind, oop, tet_rule, params = CASES[name]
    mesh = factory()
    ndof = 1 if kind == 0 else 3
    s = fea.System.from_mesh(mesh, ndof)
    try:
        if block_nodes:
            fea.fea_mesh_set_rows_block(s.handle, block_nodes)
        op = fea.make_operator(kind=kind, precision=precision, scatter=scatter, tet_rule=tet_rule, **params)
        s.A.fill_(float("nan"))                     # every entry must be written
        s.assemble(op)
        s.check()
        return s.A.cpu().numpy(), s.b.cpu().numpy(), _reference(oracle, name, mesh)
    finally:
        s.close()


@pytest.mark.parametrize("scatter", list(SCATTERS))
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_assembly_matches_oracle(oracle, name, precision, scatter):
    fea = engine()
    A, b, ref = _run_case(fea, oracle, name, precision, SCATTERS[scatter])
    tol = FP64_TOL if precision == 0 else FP32_TOL
    errA, zA = err_vs_oracle(A, ref["A"], ref["NA"])
    errb, zb = err_vs_oracle(b, ref["b"], ref["Nb"])
    assert errA <= tol, (name, precision, errA)
    assert errb <= tol, (name, precision, errb)
    assert zA <= tol and zb <= tol, (name, precision, zA, zb)


def test_inverted_element_is_reported_by_check():
    fea = engine()
    mesh = mg.hex_cube(3, 0.1, 1)
    conn = mesh.conn.copy().reshape(-1, 8)
    conn[7] = conn[7][[4, 5, 6, 7, 0, 1, 2, 3]]
    mesh.conn = conn.reshape(-1)
    s = fea.System.from_mesh(mesh, 3)
    try:
        for precision in (0, 1, 2):
            s.assemble(fea.make_operator(kind=1, precision=precision))
            with pytest.raises(fea.FeaError) as ei:
                s.check()
            assert ei.value.code == fea.FEA_ERR_INVERTED_ELEMENT
            assert "element 7" in str(ei.value)
        # the status is cleared by the check; a valid operator call afterwards still works
        s.check()
    finally:
        s.close()


def test_invalid_arguments_rejected_on_host():
    fea = engine()
    mesh = mg.hex_cube(2)
    with pytest.raises(fea.FeaError) as ei:
        bad = mesh.conn.copy(); bad[3] = mesh.n_nodes + 5
        fea.fea_mesh_upload(mesh.coords, mesh.types, mesh.conn_offsets, bad)
    assert ei.value.code == fea.FEA_ERR_ARG
    s = fea.System.from_mesh(mesh, 1)
    try:
        with pytest.raises(fea.FeaError):            # pattern built for ndof 1, elasticity needs 3
            s.assemble(fea.make_operator(kind=1))
        with pytest.raises(fea.FeaError):
            s.assemble(fea.make_operator(kind=0, tet_rule=7))
    finally:
        s.close()


@pytest.mark.parametrize("block_nodes", [1, 7, 64, 255])
@pytest.mark.parametrize("name", ["hybrid6_diffusion", "hybrid5_elasticity", "stretched_hex_elasticity"])
def test_rows_block_sizes(oracle, name, block_nodes):
    """Owner blocks of any size (one node, ragged, the default, many) give the same system."""
    fea = engine()
    A, b, ref = _run_case(fea, oracle, name, 1, scatter=3, block_nodes=block_nodes)
    errA, _ = err_vs_oracle(A, ref["A"], ref["NA"])
    errb, _ = err_vs_oracle(b, ref["b"], ref["Nb"])
    assert errA <= FP32_TOL and errb <= FP32_TOL, (errA, errb)


def test_rows_is_deterministic_and_symmetric():
    """ROWS writes every entry once with plain stores: bitwise reproducible.

    Entries whose two nodes share an owner block are computed once and written
    to both triangles (bitwise symmetric); entries between blocks are computed
    by each owner in its own order, so the matrix is symmetric to rounding.
    """
    fea = engine()
    import torch
    mesh = mg.hex_cube(9, 0.2, 4)
    s = fea.System.from_mesh(mesh, 3)
    try:
        op = fea.make_operator(kind=1, precision=1, scatter=3)
        s.assemble(op)
        A1 = s.A.clone()
        s.assemble(op)
        assert torch.equal(A1, s.A)
        import scipy.sparse as sps
        M = sps.csr_matrix((s.A.cpu().numpy(), s.col_idx.cpu().numpy(), s.row_ptr.cpu().numpy()))
        asym = abs(M - M.T).max()
        assert asym <= 1e-6 * abs(M).max()
        exact = (M - M.T).count_nonzero()
        assert exact < M.nnz // 2                     # most entries are computed once for both triangles
        info = fea.fea_rows_plan_info(s.handle)
        assert info["blocks"] >= -(-mesh.n_nodes // 64) and info["tasks"] > 0
    finally:
        s.close()


@pytest.mark.parametrize("name", ["hybrid6_diffusion", "hex10_elasticity", "kuhn16_poisson"])
def test_coloring_is_valid(name):
    """No two elements of one color class share a node (Alg. "coloring")."""
    fea = engine()
    factory, kind, _, tet_rule, params = CASES[name]
    mesh = factory()
    s = fea.System.from_mesh(mesh, 1 if kind == 0 else 3)
    try:
        s.assemble(fea.make_operator(kind=kind, scatter=fea.FEA_SCATTER_COLOR, tet_rule=tet_rule, **params))
        s.check()
        n_colors, colors = fea.fea_color_info(s.handle, mesh.n_elems)
        assert colors.min() == 0 and colors.max() == n_colors - 1
        seen = {}
        for e in range(mesh.n_elems):
            for node in mesh.element_nodes(e):
                key = (int(node), int(colors[e]))
                assert key not in seen, (e, seen.get(key))
                seen[key] = e
        assert fea.fea_assemble_launches(fea.make_operator(kind=kind, scatter=1), s.handle) >= n_colors
    finally:
        s.close()


def _tet_fan(count=70):
    """`count` tets sharing node 0 (and no other node): every element touches
    every other, so any valid coloring needs `count` colors."""
    rng = np.random.default_rng(9)
    coords = [np.zeros(3)]
    conn = []
    for k in range(count):
        d = np.array([np.cos(2 * np.pi * k / count), np.sin(2 * np.pi * k / count), 0.3 * k / count])
        base = len(coords)
        pts = [d, d + np.array([0.1, 0.0, 0.0]) + 0.01 * rng.random(3), d + np.array([0.0, 0.1, 0.1])]
        a = np.array(pts)
        if np.linalg.det(a) < 0:                      # orient every tet positively
            pts[1], pts[2] = pts[2], pts[1]
        coords += pts
        conn += [0, base, base + 1, base + 2]
    coords = np.array(coords)
    return mg.Mesh(coords=coords, types=np.zeros(count, dtype=np.uint8),
                   conn_offsets=np.arange(0, 4 * count + 1, 4, dtype=np.int64), conn=np.array(conn, dtype=np.int32))


def test_coloring_beyond_64_colors_takes_the_device_rounds(oracle):
    """Greedy coloring keeps a 64-bit mask per node; a mesh needing more colors
    is colored by Luby / Jones-Plassmann rounds on the GPU instead.  The
    coloring stays valid and the COLOR assembly matches the oracle."""
    fea = engine()
    mesh = _tet_fan(70)
    s = fea.System.from_mesh(mesh, 1)
    try:
        s.assemble(fea.make_operator(kind=0, scatter=fea.FEA_SCATTER_COLOR, precision=0, tet_rule=1, k0=1.0,
                                     k2=1.0, source=1.0))
        s.check()
        n_colors, colors = fea.fea_color_info(s.handle, mesh.n_elems)
        assert n_colors >= 70 and len(np.unique(colors)) == 70     # one element per color
        ref = oracle.assemble(mesh, 0, tet_rule=1, k0=1.0, k2=1.0, source=1.0)
        errA, zA = err_vs_oracle(s.A.cpu().numpy(), ref["A"], ref["NA"])
        errb, zb = err_vs_oracle(s.b.cpu().numpy(), ref["b"], ref["Nb"])
        assert max(errA, errb, zA, zb) <= FP64_TOL
    finally:
        s.close()
