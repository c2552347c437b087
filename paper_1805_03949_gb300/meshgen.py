"""Seeded synthetic meshes: the inputs of every test and benchmark.

This module only builds input arrays (node coordinates, element types and
connectivity, displacement fields).  It holds none of the finite-element
arithmetic (no shape functions, quadrature, Jacobians or element matrices), so
that both the CUDA engine and the CPU oracle can consume its output without
sharing any of the method's code.

The paper's own workloads (the 17.7 M-element respiratory mesh of Sec. 2.1.5
and the 31.5 M-element Iter mesh of Sec. 2.2.2) are not available; the meshes
below are synthetic stand-ins with the element types and sizes of those
problems:

* ``kuhn_tet_cube(n)``        -- unit cube, n^3 cells, 6 Kuhn tetrahedra per cell
* ``hex_cube(n, jitter, seed)`` -- unit cube, n^3 trilinear hexahedra, interior
  nodes moved by U(-jitter*h, +jitter*h) per coordinate
* ``hybrid_cube(n, seed)``    -- unit cube split into four type zones (tet4 40 %,
  pyr5 10 %, prism6 20 %, hex8 30 % of the elements)
* ``batch_meshes(count, seed)`` -- many tet4/hex8 boxes of log-uniform size
* ``fourier_displacement(...)`` -- smooth nodal displacement field (sum of
  sine modes) used as the state of the elastoplastic operator
* ``mlp_initial_params(n_in, seed)`` -- seeded initial weights of the cost model

Element type codes and local node orders (shared convention of the C-ABI):

* 0 tet4   : reference simplex, node 0 at the origin, nodes 1..3 on the axes
* 1 pyr5   : base square [-1,1]^2 at zeta=0 counter-clockwise seen from the
  apex, apex (0,0,1) last
* 2 prism6 : bottom triangle (counter-clockwise seen from the top) then the
  top triangle in the same order
* 3 hex8   : (000,100,110,010,001,101,111,011) lexicographic-VTK order
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TET4, PYR5, PRISM6, HEX8 = 0, 1, 2, 3
NODES_PER_TYPE = {TET4: 4, PYR5: 5, PRISM6: 6, HEX8: 8}
TYPE_NAMES = {TET4: "tet4", PYR5: "pyr5", PRISM6: "prism6", HEX8: "hex8"}


@dataclass
class Mesh:
    """A mesh in the array layout the engine's ``fea_mesh_upload`` takes.

    coords       float64 [n_nodes, 3]   xyz per node
    types        uint8   [n_elems]      element type code
    conn_offsets int64   [n_elems + 1]  start of each element in ``conn``
    conn         int32   [conn_offsets[-1]] node ids, local order per type
    """

    coords: np.ndarray
    types: np.ndarray
    conn_offsets: np.ndarray
    conn: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.types.shape[0])

    def element_nodes(self, e: int) -> np.ndarray:
        return self.conn[self.conn_offsets[e]:self.conn_offsets[e + 1]]


def _uniform_mesh(coords, etype, conn2d, meta) -> Mesh:
    conn2d = np.ascontiguousarray(conn2d, dtype=np.int32)
    ne, nn = conn2d.shape
    offsets = np.arange(ne + 1, dtype=np.int64) * nn
    types = np.full(ne, etype, dtype=np.uint8)
    return Mesh(np.ascontiguousarray(coords, dtype=np.float64), types, offsets,
                conn2d.reshape(-1), meta)


def _lattice_coords(nx, ny, nz):
    """Nodes of an nx*ny*nz-cell box on [0,1]^3, x fastest: id = i + (nx+1)(j + (ny+1)k)."""
    x = np.arange(nx + 1, dtype=np.float64) / nx
    y = np.arange(ny + 1, dtype=np.float64) / ny
    z = np.arange(nz + 1, dtype=np.float64) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _cell_origins(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


# Kuhn split of the unit cube: tet p = (v, v+e_a, v+e_a+e_b, v+(1,1,1)) for
# each permutation (a,b,c) of the axes in lexicographic order.  Its signed
# volume has the sign of the permutation, so for odd permutations the last two
# nodes are swapped to keep every tetrahedron positively oriented.
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
_PERM_ODD = [False, True, True, False, False, True]


def _kuhn_offsets():
    """Corner offsets (dx,dy,dz) of the 6 Kuhn tets of a cell, positively oriented."""
    out = []
    for perm, odd in zip(_PERMS, _PERM_ODD):
        p0 = np.zeros(3, dtype=np.int64)
        p1 = p0.copy(); p1[perm[0]] = 1
        p2 = p1.copy(); p2[perm[1]] = 1
        p3 = np.ones(3, dtype=np.int64)
        tet = [p0, p1, p2, p3]
        if odd:
            tet = [p0, p1, p3, p2]
        out.append(np.stack(tet))
    return np.stack(out)  # [6, 4, 3]


_HEX_OFFSETS = np.array([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                         (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)], dtype=np.int64)


def kuhn_tet_cube(n: int, nx: int | None = None, ny: int | None = None,
                  nz: int | None = None) -> Mesh:
    """Unit cube of n^3 cells (or nx*ny*nz), each split into 6 Kuhn tets; no randomness.

    Elements are numbered cell by cell (x fastest), 6 per cell.
    """
    nx = nx or n; ny = ny or n; nz = nz or n
    coords = _lattice_coords(nx, ny, nz)
    ci, cj, ck = _cell_origins(nx, ny, nz)
    off = _kuhn_offsets()
    ii = ci[:, None, None] + off[None, :, :, 0]
    jj = cj[:, None, None] + off[None, :, :, 1]
    kk = ck[:, None, None] + off[None, :, :, 2]
    node = ii + (nx + 1) * (jj + (ny + 1) * kk)
    conn = node.reshape(-1, 4)
    return _uniform_mesh(coords, TET4, conn, {"kind": "kuhn_tet", "n": (nx, ny, nz)})


def hex_cube(n: int, jitter: float = 0.0, seed: int | None = None,
             nx: int | None = None, ny: int | None = None, nz: int | None = None) -> Mesh:
    """Unit cube of n^3 hex8 cells; interior nodes jittered by U(-jitter*h, jitter*h).

    The jitter is drawn for every node and coordinate, in node order, from
    ``numpy.random.Generator(PCG64(seed))`` and applied to interior nodes only
    (h is the cell size along that axis).
    """
    nx = nx or n; ny = ny or n; nz = nz or n
    coords = _lattice_coords(nx, ny, nz)
    if jitter:
        rng = np.random.Generator(np.random.PCG64(seed))
        d = rng.uniform(-jitter, jitter, size=coords.shape)
        d *= np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        interior = ((i > 0) & (i < nx) & (j > 0) & (j < ny) & (k > 0) & (k < nz)).ravel()
        coords[interior] += d[interior]
    ci, cj, ck = _cell_origins(nx, ny, nz)
    o = _HEX_OFFSETS
    node = (ci[:, None] + o[None, :, 0]) + (nx + 1) * ((cj[:, None] + o[None, :, 1])
                                                       + (ny + 1) * (ck[:, None] + o[None, :, 2]))
    return _uniform_mesh(coords, HEX8, node, {"kind": "hex", "n": (nx, ny, nz),
                                              "jitter": jitter, "seed": seed})


# ---------------------------------------------------------------------------
# hybrid mesh: four type zones on a fine lattice of half-cells
# ---------------------------------------------------------------------------

# Per-zone cell templates in half-cell units (a cell spans 0..2 per axis).
def _hybrid_templates():
    tets = [[tuple(2 * c) for c in t] for t in _kuhn_offsets()]
    # 6 pyramids: base = a cell face, apex = cell centre (1,1,1); base listed
    # counter-clockwise seen from the apex.
    pyr_bases = [
        [(0, 0, 0), (2, 0, 0), (2, 2, 0), (0, 2, 0)],   # z = 0
        [(0, 0, 2), (0, 2, 2), (2, 2, 2), (2, 0, 2)],   # z = 2
        [(0, 0, 0), (0, 2, 0), (0, 2, 2), (0, 0, 2)],   # x = 0
        [(2, 0, 0), (2, 0, 2), (2, 2, 2), (2, 2, 0)],   # x = 2
        [(0, 0, 0), (0, 0, 2), (2, 0, 2), (2, 0, 0)],   # y = 0
        [(0, 2, 0), (2, 2, 0), (2, 2, 2), (0, 2, 2)],   # y = 2
    ]
    pyrs = [b + [(1, 1, 1)] for b in pyr_bases]
    # 2 prisms split by the plane through the (0,0)-(1,1) face diagonal (the
    # same diagonal as the Kuhn split), extruded along z.
    tri = [[(0, 0), (2, 0), (2, 2)], [(0, 0), (2, 2), (0, 2)]]
    prisms = [[(x, y, 0) for x, y in t] + [(x, y, 2) for x, y in t] for t in tri]
    # 2x2x2 refinement into hexes.
    hexes = []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                hexes.append([(dx + a, dy + b, dz + c) for a, b, c in _HEX_OFFSETS.tolist()])
    return {TET4: tets, PYR5: pyrs, PRISM6: prisms, HEX8: hexes}


_HYBRID_PER_CELL = {TET4: 6, PYR5: 6, PRISM6: 2, HEX8: 8}
HYBRID_FRACTIONS = {TET4: 0.4, PYR5: 0.1, PRISM6: 0.2, HEX8: 0.3}


def hybrid_zone_cells(n: int) -> dict:
    """Cells per zone so the element fractions are 40/10/20/30 % (largest remainder)."""
    cells = n ** 3
    denom = sum(HYBRID_FRACTIONS[t] / _HYBRID_PER_CELL[t] for t in (TET4, PYR5, PRISM6, HEX8))
    exact = {t: cells * (HYBRID_FRACTIONS[t] / _HYBRID_PER_CELL[t]) / denom for t in HYBRID_FRACTIONS}
    base = {t: int(np.floor(v)) for t, v in exact.items()}
    rem = cells - sum(base.values())
    for t in sorted(exact, key=lambda t: (-(exact[t] - base[t]), t))[:rem]:
        base[t] += 1
    return base


def hybrid_cube(n: int = 100, seed: int = 3) -> Mesh:
    """Unit cube of n^3 cells split into tet4/pyr5/prism6/hex8 zones.

    Zones are quantiles of a smooth seeded field (6 sine modes) at the cell
    centres, ties broken by cell id.  Zone interfaces are non-conforming
    (hanging nodes); every element is affine or trilinear and positively
    oriented.  Elements are emitted cell by cell (x fastest), keeping spatial
    locality.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    kvec = rng.integers(1, 4, size=(6, 3)).astype(np.float64)
    phase = rng.uniform(0.0, 2 * np.pi, size=6)
    amp = rng.uniform(0.5, 1.0, size=6)
    ci, cj, ck = _cell_origins(n, n, n)
    centres = (np.stack([ci, cj, ck], axis=1) + 0.5) / n
    fieldv = np.zeros(len(ci))
    for m in range(6):
        fieldv += amp[m] * np.sin(2 * np.pi * centres @ kvec[m] + phase[m])
    order = np.lexsort((np.arange(len(ci)), fieldv))
    counts = hybrid_zone_cells(n)
    zone = np.empty(len(ci), dtype=np.int64)
    start = 0
    for t in (TET4, PYR5, PRISM6, HEX8):
        zone[order[start:start + counts[t]]] = t
        start += counts[t]

    return _template_mesh(n, zone, {"kind": "hybrid", "n": n, "seed": seed, "zone_cells": counts})


def _template_mesh(n: int, zone: np.ndarray, meta: dict, jitter: float = 0.0, seed=None) -> Mesh:
    """Fill cell c (x fastest) of an n^3 box with the template of type zone[c]."""
    ci, cj, ck = _cell_origins(n, n, n)
    tmpl = _hybrid_templates()
    m = 2 * n + 1
    per_cell = np.array([_HYBRID_PER_CELL[t] for t in range(4)])[zone]
    nn_of = np.array([NODES_PER_TYPE[t] for t in range(4)])
    # element list in cell order; within a cell the template order
    elem_cell = np.repeat(np.arange(len(ci)), per_cell)
    elem_type = np.repeat(zone, per_cell)
    elem_local = np.arange(len(elem_cell)) - np.repeat(np.cumsum(per_cell) - per_cell, per_cell)
    nn = nn_of[elem_type]
    offsets = np.zeros(len(elem_cell) + 1, dtype=np.int64)
    np.cumsum(nn, out=offsets[1:])
    fine = np.empty(offsets[-1], dtype=np.int64)
    for t in range(4):
        sel = np.nonzero(elem_type == t)[0]
        if len(sel) == 0:
            continue
        T = np.array(tmpl[t], dtype=np.int64)                     # [per_cell, nn, 3]
        loc = T[elem_local[sel]]                                   # [ne, nn, 3]
        c = elem_cell[sel]
        I = 2 * ci[c][:, None] + loc[:, :, 0]
        J = 2 * cj[c][:, None] + loc[:, :, 1]
        K = 2 * ck[c][:, None] + loc[:, :, 2]
        f = I + m * (J + m * K)
        idx = offsets[sel][:, None] + np.arange(NODES_PER_TYPE[t])[None, :]
        fine[idx] = f
    used, conn = np.unique(fine, return_inverse=True)
    I = used % m
    J = (used // m) % m
    K = used // (m * m)
    coords = np.stack([I, J, K], axis=1).astype(np.float64) / (2 * n)
    if jitter:
        rng = np.random.Generator(np.random.PCG64(seed))
        d = rng.uniform(-jitter, jitter, size=coords.shape) / (2 * n)
        interior = (I > 0) & (I < m - 1) & (J > 0) & (J < m - 1) & (K > 0) & (K < m - 1)
        coords[interior] += d[interior]
    return Mesh(coords, elem_type.astype(np.uint8), offsets, conn.astype(np.int32), meta)


def template_cube(n: int, etype: int, jitter: float = 0.0, seed=None) -> Mesh:
    """Conforming single-type mesh: every cell of an n^3 box gets the template of ``etype``.

    tet4: 6 Kuhn tets; pyr5: 6 pyramids around a cell-centre node; prism6: 2
    prisms; hex8: 2x2x2 refinement.  Interior nodes move by
    U(-jitter, jitter) half-cells per coordinate (PCG64(seed)).
    """
    zone = np.full(n ** 3, etype, dtype=np.int64)
    return _template_mesh(n, zone, {"kind": "template", "n": n, "type": etype, "jitter": jitter,
                                    "seed": seed}, jitter, seed)


# ---------------------------------------------------------------------------
# batched meshes and displacement fields
# ---------------------------------------------------------------------------

def _box_dims(cells: float):
    n = max(1, int(round(cells ** (1.0 / 3.0))))
    nz = max(1, int(round(cells / (n * n))))
    return n, n, nz


def batch_meshes(count: int = 256, seed: int = 5, lo: float = 1e3, hi: float = 2e5,
                 jitter: float = 0.2) -> list:
    """``count`` independent tet4/hex8 boxes, sizes log-uniform in [lo, hi] elements.

    Type is tet4 or hex8 with probability 1/2; box dims are the integer
    triple closest to a cube with that many elements (tet: 6 per cell); hex
    boxes are jittered like ``hex_cube`` with seed ``seed*1000 + i``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))
    kinds = rng.integers(0, 2, size=count)
    out = []
    for i in range(count):
        if kinds[i] == 0:
            nx, ny, nz = _box_dims(sizes[i] / 6.0)
            msh = kuhn_tet_cube(0, nx, ny, nz)
        else:
            nx, ny, nz = _box_dims(sizes[i])
            msh = hex_cube(0, jitter, seed * 1000 + i, nx, ny, nz)
        msh.meta["target_elems"] = float(sizes[i])
        out.append(msh)
    return out


def fourier_displacement(coords: np.ndarray, amplitude: float, seed: int = 4,
                         modes: int = 8) -> np.ndarray:
    """u(x) = A * sum_m a_m sin(2 pi k_m . x + phi_m), k_m in {1..4}^3, |a_m| = 1.

    Drawn from ``numpy.random.Generator(PCG64(seed))`` in the order k, a, phi.
    Returns float64 [n_nodes, 3].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.integers(1, 5, size=(modes, 3)).astype(np.float64)
    a = rng.normal(size=(modes, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    phi = rng.uniform(0.0, 2 * np.pi, size=modes)
    u = np.zeros_like(coords)
    for m in range(modes):
        u += np.sin(2 * np.pi * coords @ k[m] + phi[m])[:, None] * a[m][None, :]
    return amplitude * u


def j2_workload(n: int = 96, amplitude: float = 1.0, seed_mesh: int = 6, seed_u: int = 4):
    """Elastoplastic hex8 workload: n^3 jittered cube (+-0.2h, PCG64(seed_mesh)) and the
    nodal displacement field fourier_displacement(coords, amplitude, seed_u).

    The load is applied in two steps, 0.5 u then u; the amplitude that makes
    about 30% of the Gauss points yield in the second step is a stored fixture.
    """
    mesh = hex_cube(n, 0.2, seed_mesh)
    return mesh, fourier_displacement(mesh.coords, amplitude, seed=seed_u)


def partition_elements(mesh: Mesh, parts: int):
    """Element partition into `parts` subdomains of consecutive element-centroid
    z order (slabs), as the partial-row decomposition of Sec. 3.1 uses them.

    Returns a list of (submesh, glob): the submesh has the elements of one part
    with its own node numbering (nodes in increasing global id), glob [n_local]
    its local -> global node ids; and the multiplicity of every global node
    (how many parts hold it).
    """
    off = mesh.conn_offsets
    nn = np.diff(off)
    cz = np.zeros(mesh.n_elems)
    np.add.at(cz, np.repeat(np.arange(mesh.n_elems), nn), mesh.coords[mesh.conn, 2])
    cz /= nn
    order = np.argsort(cz, kind="stable")
    chunks = np.array_split(order, parts)
    mult = np.zeros(mesh.n_nodes, dtype=np.int32)
    out = []
    for ids in chunks:
        ids = np.sort(ids)
        cnt = nn[ids]
        starts = off[ids]
        idx = np.repeat(starts, cnt) + (np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt))
        gconn = mesh.conn[idx]
        glob = np.unique(gconn).astype(np.int32)
        mult[glob] += 1
        lconn = np.searchsorted(glob, gconn).astype(np.int32)
        coff = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
        sub = Mesh(mesh.coords[glob].copy(), mesh.types[ids].copy(), coff, lconn, dict(mesh.meta, part_of=len(out)))
        out.append((sub, glob))
    return out, mult


def mlp_initial_params(n_in: int, seed: int = 6, hidden: int = 32) -> np.ndarray:
    """Initial parameters of the cost model (n_in -> hidden tanh -> hidden tanh
    -> 1), in the C-ABI's order W1 [hidden][n_in], b1, W2 [hidden][hidden], b2,
    w3 [hidden], b3: Xavier-uniform weights (bound sqrt(6 / (fan_in +
    fan_out))) drawn from PCG64(seed) in that order, zero biases.  A seeded
    input like the meshes, for the engine and the oracle alike."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def lim(fan_in, fan_out):
        return np.sqrt(6.0 / (fan_in + fan_out))

    W1 = rng.uniform(-lim(n_in, hidden), lim(n_in, hidden), (hidden, n_in))
    W2 = rng.uniform(-lim(hidden, hidden), lim(hidden, hidden), (hidden, hidden))
    w3 = rng.uniform(-lim(hidden, 1), lim(hidden, 1), hidden)
    return np.concatenate([W1.ravel(), np.zeros(hidden), W2.ravel(), np.zeros(hidden), w3, [0.0]])
