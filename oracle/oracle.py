"""Python access to the plain FP64 CPU oracle (``fea_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module; the engine never
does.  The oracle shares no code with the CUDA engine: it is compiled from
its own C source with gcc, and its inputs are plain numpy arrays (typically
from ``paper_1805_03949_gb300.meshgen``).

Every function follows the assembly loop of the paper (Alg. "sequential
assembly", Sec. 2.1.1) over the square local CSR system of Sec. 3.1; see the
header of ``fea_oracle.c`` for the element formulations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fea_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OP_DIFFUSION, OP_ELASTICITY = 0, 1
NODES = {0: 4, 1: 5, 2: 6, 3: 8}

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [_SRC] + [os.path.join(_HERE, f) for f in sorted(os.listdir(_HERE))
                     if f.endswith(".c") and f != "fea_oracle.c"]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp] + srcs + ["-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    """The compiled oracle (built on first use), with its C signatures declared."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.oracle_pattern.restype = _i64
            _lib.oracle_pattern.argtypes = [_i64, _i64, _p, _p, _p, _p, _p, _p]
            _lib.oracle_expand_pattern.restype = None
            _lib.oracle_expand_pattern.argtypes = [_i64, _i32, _p, _p, _p, _p]
            _lib.oracle_assemble.restype = _i64
            _lib.oracle_assemble.argtypes = [_i64, _i64, _p, _p, _p, _p, _i32, _i32, _p, _p, _p, _p, _p, _p, _p, _p]
            _lib.oracle_assemble_rows.restype = _i64
            _lib.oracle_assemble_rows.argtypes = [_i64, _i64, _p, _p, _p, _p, _i32, _i32, _p, _i64, _p, _i64,
                                                  _p, _p, _p, _p, _p, _p, _p]
            _lib.oracle_element.restype = _i32
            _lib.oracle_element.argtypes = [_i32, _i32, _i32, _p, _p, _p, _p, _p, _p, _p]
            _lib.oracle_quadrature.restype = _i32
            _lib.oracle_quadrature.argtypes = [_i32, _i32, _p, _p]
            _lib.oracle_shape.restype = _i32
            _lib.oracle_shape.argtypes = [_i32, _p, _p, _p]
            for name, (rt, at) in _extra_signatures().items():
                f = getattr(_lib, name)
                f.restype = rt
                f.argtypes = at
        return _lib


def _extra_signatures():
    return {
        "oracle_j2_point": (_i32, [_p, _p, _p, ctypes.c_double, _p, _p, _p, _p, _p, _p]),
        "oracle_j2_element": (_i32, [_i32, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p]),
        "oracle_j2_assemble": (_i64, [_i64, _i64, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p]),
        "oracle_j2_sweep": (_i64, [_i64, _p, _p, _p, _p, _p, _p, ctypes.c_double, _p, _p, _p, _p, _p]),
        "oracle_nh_point": (_i32, [_p, _p, _p, _p, _p]),
        "oracle_nh_element": (_i32, [_i32, _p, _p, _p, _p, _p, _p, _p, _p]),
        "oracle_nh_assemble": (_i64, [_i64, _i64, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p]),
    }


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class InvertedElement(RuntimeError):
    """det J <= 0 at a quadrature point (the element id, or -1 for a single element)."""
    def __init__(self, elem):
        super().__init__(f"element {elem} has detJ <= 0 at a quadrature point")
        self.elem = elem


def op_params(op: int, **kw) -> np.ndarray:
    """Operator parameters in the oracle's order: diffusion (k0, k2, f); elasticity (E, nu, f_x, f_y, f_z)."""
    if op == OP_DIFFUSION:
        return np.array([kw.get("k0", 1.0), kw.get("k2", 0.0), kw.get("source", 1.0)], dtype=np.float64)
    f = kw.get("body_force", (1.0, 1.0, 1.0))
    return np.array([kw.get("young", 1.0), kw.get("poisson", 0.3), f[0], f[1], f[2]], dtype=np.float64)


def quadrature(etype: int, tet_rule: int = 1):
    """Reference points [nq, 3] and weights [nq] of the element type's rule (tet_rule 0: centroid, 1: 4-point)."""
    pts = np.zeros((8, 3)); w = np.zeros(8)
    nq = lib().oracle_quadrature(etype, tet_rule, _ptr(pts), _ptr(w))
    return pts[:nq].copy(), w[:nq].copy()


def shape(etype: int, p):
    """N [nn] and dN/dxi [nn, 3] of the element type at reference point p."""
    p = _c(p, np.float64)
    N = np.zeros(8); dN = np.zeros((8, 3))
    nn = lib().oracle_shape(etype, _ptr(p), _ptr(N), _ptr(dN))
    return N[:nn].copy(), dN[:nn].copy()


def element(etype: int, X, op: int = OP_DIFFUSION, tet_rule: int = 1, **kw):
    """Element matrix, RHS and magnitude sums of one element with node coordinates X [nn,3]."""
    X = _c(X, np.float64)
    d = 1 if op == OP_DIFFUSION else 3
    n = NODES[etype] * d
    Ae = np.zeros((n, n)); be = np.zeros(n); Se = np.zeros((n, n)); Sb = np.zeros(n); Ne = np.zeros((n, n))
    params = op_params(op, **kw)
    rc = lib().oracle_element(etype, tet_rule, op, _ptr(params), _ptr(X), _ptr(Ae), _ptr(be), _ptr(Se), _ptr(Sb),
                              _ptr(Ne))
    if rc:
        raise InvertedElement(-1)
    if kw.get("with_norm"):
        return Ae, be, Se, Sb, Ne
    return Ae, be, Se, Sb


def pattern(mesh, ndof: int = 1):
    """CSR pattern (scalar, ndof interleaved dofs per node) and the node rank map.

    Returns (row_ptr int64 [n*ndof+1], col_idx int32 [nnz], node_map int32
    [sum n_e^2]).  node_map[off(e) + a*n_e + b] is the rank k of node
    conn[e][b] among the sorted neighbours of node conn[e][a]; the scalar entry
    of (dof d*i+c, dof d*j+c') sits at row_ptr[d*i+c] + d*k + c'.
    """
    L = lib()
    types = _c(mesh.types, np.uint8); off = _c(mesh.conn_offsets, np.int64); conn = _c(mesh.conn, np.int32)
    n = mesh.n_nodes
    rp = np.zeros(n + 1, dtype=np.int64)
    nnz = L.oracle_pattern(n, mesh.n_elems, _ptr(types), _ptr(off), _ptr(conn), _ptr(rp), None, None)
    if nnz < 0:
        raise ValueError("bad mesh")
    col = np.zeros(nnz, dtype=np.int32)
    nn = np.diff(off)
    nmap = np.zeros(int((nn * nn).sum()), dtype=np.int32)
    L.oracle_pattern(n, mesh.n_elems, _ptr(types), _ptr(off), _ptr(conn), _ptr(rp), _ptr(col), _ptr(nmap))
    if ndof == 1:
        return rp, col, nmap
    rps = np.zeros(n * ndof + 1, dtype=np.int64)
    cols = np.zeros(nnz * ndof * ndof, dtype=np.int32)
    L.oracle_expand_pattern(n, ndof, _ptr(rp), _ptr(col), _ptr(rps), _ptr(cols))
    return rps, cols, nmap


def assemble(mesh, op: int = OP_DIFFUSION, tet_rule: int = 1, pat=None, **kw):
    """Assemble A (CSR values) and b in element-index order, with magnitude sums.

    Returns dict(row_ptr, col_idx, node_map, A, b, SA, Sb, NA): SA/Sb the
    componentwise magnitude sums, NA the normwise scale (Nb = Sb).
    """
    d = 1 if op == OP_DIFFUSION else 3
    if pat is None:
        pat = pattern(mesh, d)
    rps, cols, nmap = pat
    A = np.zeros(cols.shape[0]); SA = np.zeros_like(A); NA = np.zeros_like(A)
    b = np.zeros(mesh.n_nodes * d); Sb = np.zeros_like(b)
    params = op_params(op, **kw)
    types = _c(mesh.types, np.uint8); off = _c(mesh.conn_offsets, np.int64); conn = _c(mesh.conn, np.int32)
    coords = _c(mesh.coords, np.float64)
    rc = lib().oracle_assemble(mesh.n_nodes, mesh.n_elems, _ptr(types), _ptr(off), _ptr(conn), _ptr(coords),
                               op, tet_rule, _ptr(params), _ptr(rps), _ptr(nmap),
                               _ptr(A), _ptr(b), _ptr(SA), _ptr(Sb), _ptr(NA))
    if rc < 0:
        raise InvertedElement(-rc - 1)
    return dict(row_ptr=rps, col_idx=cols, node_map=nmap, A=A, b=b, SA=SA, Sb=Sb, NA=NA, Nb=Sb)


def assemble_rows(mesh, nodes, op: int = OP_DIFFUSION, tet_rule: int = 1, max_cols: int = 512, **kw):
    """All dof rows of the requested nodes, summed over every element in index order.

    Returns a list with, per node, dict(cols (node neighbours), vals [d, deg*d],
    svals, b [d], sb [d]).
    """
    d = 1 if op == OP_DIFFUSION else 3
    req = _c(nodes, np.int32)
    r = len(req)
    cols = np.zeros((r, max_cols), dtype=np.int32)
    deg = np.zeros(r, dtype=np.int64)
    vals = np.zeros(r * max_cols * d * d); svals = np.zeros_like(vals); nvals = np.zeros_like(vals)
    bv = np.zeros(r * d); sbv = np.zeros_like(bv)
    params = op_params(op, **kw)
    types = _c(mesh.types, np.uint8); off = _c(mesh.conn_offsets, np.int64); conn = _c(mesh.conn, np.int32)
    coords = _c(mesh.coords, np.float64)
    rc = lib().oracle_assemble_rows(mesh.n_nodes, mesh.n_elems, _ptr(types), _ptr(off), _ptr(conn), _ptr(coords),
                                    op, tet_rule, _ptr(params), r, _ptr(req), max_cols, _ptr(cols), _ptr(deg),
                                    _ptr(vals), _ptr(svals), _ptr(bv), _ptr(sbv), _ptr(nvals))
    if rc == -1:
        raise ValueError("row wider than max_cols")
    if rc < 0:
        raise InvertedElement(-rc - 1)
    out = []
    for t in range(r):
        k = int(deg[t])
        base = t * max_cols * d * d
        out.append(dict(cols=cols[t, :k].copy(),
                        vals=vals[base:base + d * k * d].reshape(d, k * d).copy(),
                        svals=svals[base:base + d * k * d].reshape(d, k * d).copy(),
                        nvals=nvals[base:base + d * k * d].reshape(d, k * d).copy(),
                        b=bv[t * d:(t + 1) * d].copy(), sb=sbv[t * d:(t + 1) * d].copy()))
    return out


# ---------------------------------------------------------------------------
# J2 plasticity with Voce hardening (j2_oracle.c)
# ---------------------------------------------------------------------------

class NoConvergence(RuntimeError):
    """The return map needed more than max_iter Newton updates."""


J2_DEFAULTS = dict(young=1.0, poisson=0.3, sigma0=1e-3, sigma_inf=3e-3, delta=300.0, hardening=1e-2,
                   tol_g=1e-13, tol_step=1e-15, max_iter=12)


def j2_params(**kw) -> np.ndarray:
    """Material and Newton parameters in the oracle's order (defaults: those of the 96^3 elastoplastic hex workload)."""
    p = dict(J2_DEFAULTS, **kw)
    return np.array([p["young"], p["poisson"], p["sigma0"], p["sigma_inf"], p["delta"], p["hardening"],
                     p["tol_g"], p["tol_step"], p["max_iter"]], dtype=np.float64)


def j2_point(eps, eps_p_n=None, alpha_n=0.0, **kw):
    """Radial return at one point: eps, eps_p tensor components (xx, yy, zz, xy, yz, xz).

    Returns dict(sigma [6], D [6, 6] on engineering strain, eps_p [6], alpha,
    iters, yielded).
    """
    prm = j2_params(**kw)
    eps = _c(eps, np.float64)
    epn = _c(np.zeros(6) if eps_p_n is None else eps_p_n, np.float64)
    sig = np.zeros(6); D = np.zeros(36); ep = np.zeros(6)
    al = ctypes.c_double(); it = ctypes.c_int(); yl = ctypes.c_int()
    rc = lib().oracle_j2_point(_ptr(prm), _ptr(eps), _ptr(epn), float(alpha_n), _ptr(sig), _ptr(D), _ptr(ep),
                               ctypes.byref(al), ctypes.byref(it), ctypes.byref(yl))
    if rc:
        raise NoConvergence("return map did not converge")
    return dict(sigma=sig, D=D.reshape(6, 6), eps_p=ep, alpha=al.value, iters=it.value, yielded=yl.value)


def j2_element(etype, X, U, state_n=None, **kw):
    """Tangent, internal force and normwise scales of one element (4-point tet rule)."""
    prm = j2_params(**kw)
    X = _c(X, np.float64); U = _c(U, np.float64)
    n = 3 * NODES[etype]
    Ae = np.zeros((n, n)); be = np.zeros(n); Ne = np.zeros((n, n)); Nb = np.zeros(n)
    st = np.zeros((8, 7)); it = np.zeros(8, dtype=np.int32); yl = np.zeros(8, dtype=np.int32)
    sn = None if state_n is None else _c(state_n, np.float64)
    rc = lib().oracle_j2_element(etype, _ptr(prm), _ptr(X), _ptr(U), _ptr(sn), _ptr(Ae), _ptr(be), _ptr(Ne),
                                 _ptr(Nb), _ptr(st), _ptr(it), _ptr(yl))
    if rc == 1:
        raise InvertedElement(-1)
    if rc == 2:
        raise NoConvergence("return map did not converge")
    return dict(A=Ae, b=be, NA=Ne, Nb=Nb, state=st, iters=it, yielded=yl)


def j2_assemble(mesh, U, state_n=None, pat=None, **kw):
    """Tangent matrix and internal force of the whole mesh (3 dofs per node), element-index order.

    U: [n_nodes, 3] displacements; state_n: [E, 8, 7] (None = virgin).
    Returns dict(row_ptr, col_idx, node_map, A, b, NA, Nb, state [E, 8, 7],
    iters [E, 8], yielded [E, 8]).
    """
    if pat is None:
        pat = pattern(mesh, 3)
    rps, cols, nmap = pat
    prm = j2_params(**kw)
    E = mesh.n_elems
    A = np.zeros(cols.shape[0]); NA = np.zeros_like(A)
    b = np.zeros(mesh.n_nodes * 3); Nb = np.zeros_like(b)
    st = np.zeros((E, 8, 7)); it = np.zeros((E, 8), dtype=np.int32); yl = np.zeros((E, 8), dtype=np.uint8)
    sn = None if state_n is None else _c(state_n, np.float64)
    types = _c(mesh.types, np.uint8); off = _c(mesh.conn_offsets, np.int64); conn = _c(mesh.conn, np.int32)
    coords = _c(mesh.coords, np.float64); U = _c(U, np.float64)
    rc = lib().oracle_j2_assemble(mesh.n_nodes, E, _ptr(types), _ptr(off), _ptr(conn), _ptr(coords), _ptr(prm),
                                  _ptr(U), _ptr(sn), _ptr(rps), _ptr(nmap), _ptr(A), _ptr(b), _ptr(NA), _ptr(Nb),
                                  _ptr(st), _ptr(it), _ptr(yl))
    if rc < 0 and -rc <= E:
        raise InvertedElement(-rc - 1)
    if rc < 0:
        raise NoConvergence(f"return map of element {-rc - E - 1} did not converge")
    return dict(row_ptr=rps, col_idx=cols, node_map=nmap, A=A, b=b, NA=NA, Nb=Nb, state=st, iters=it, yielded=yl)


def j2_sweep(mesh, U, scale=1.0, state_n=None, want_state=False, **kw):
    """Count the yielding Gauss points at displacement scale*U (no assembly); optionally the new state."""
    prm = j2_params(**kw)
    types = _c(mesh.types, np.uint8); off = _c(mesh.conn_offsets, np.int64); conn = _c(mesh.conn, np.int32)
    coords = _c(mesh.coords, np.float64); U = _c(U, np.float64)
    st = np.zeros((mesh.n_elems, 8, 7)) if want_state else None
    sn = None if state_n is None else _c(state_n, np.float64)
    n = lib().oracle_j2_sweep(mesh.n_elems, _ptr(types), _ptr(off), _ptr(conn), _ptr(coords), _ptr(prm), _ptr(U),
                              float(scale), _ptr(sn), _ptr(st), None, None, None)
    if n < 0:
        raise NoConvergence("inverted element or failed return map")
    return (int(n), st) if want_state else int(n)


def j2_points(mesh, U, state_n=None, **kw):
    """The element-wise loop: per (element, point slot) the new state [E,8,7], stress [E,8,6],
    Newton iteration counts and yield flags [E,8] (slots past the rule's points stay 0)."""
    prm = j2_params(**kw)
    E = mesh.n_elems
    types = _c(mesh.types, np.uint8); off = _c(mesh.conn_offsets, np.int64); conn = _c(mesh.conn, np.int32)
    coords = _c(mesh.coords, np.float64); U = _c(U, np.float64)
    st = np.zeros((E, 8, 7)); sig = np.zeros((E, 8, 6))
    it = np.zeros((E, 8), dtype=np.int32); yl = np.zeros((E, 8), dtype=np.uint8)
    sn = None if state_n is None else _c(state_n, np.float64)
    n = lib().oracle_j2_sweep(E, _ptr(types), _ptr(off), _ptr(conn), _ptr(coords), _ptr(prm), _ptr(U), 1.0, _ptr(sn),
                              _ptr(st), _ptr(sig), _ptr(it), _ptr(yl))
    if n < 0:
        raise NoConvergence("inverted element or failed return map")
    return dict(state=st, stress=sig, iters=it, yielded=yl, n_yielded=int(n))


# ---------------------------------------------------------------------------
# finite-strain neo-Hookean solid (nh_oracle.c)
# ---------------------------------------------------------------------------

def nh_params(young=1.0, poisson=0.3, mass=0.0) -> np.ndarray:
    """E, nu and the Newmark mass coefficient m = rho0 / (beta dt^2)."""
    return np.array([young, poisson, mass], dtype=np.float64)


def nh_point(F, **kw):
    """First Piola-Kirchhoff stress P [3, 3], tangent dP/dF [3, 3, 3, 3] and energy density at F."""
    prm = nh_params(**kw)
    F = _c(F, np.float64)
    P = np.zeros(9); At = np.zeros(81); psi = ctypes.c_double()
    if lib().oracle_nh_point(_ptr(prm), _ptr(F), _ptr(P), _ptr(At), ctypes.byref(psi)):
        raise InvertedElement(-1)
    return dict(P=P.reshape(3, 3), A=At.reshape(3, 3, 3, 3), psi=psi.value)


def nh_element(etype, X, U, **kw):
    """Jacobian, internal force, normwise scales and stored energy of one element."""
    prm = nh_params(**kw)
    X = _c(X, np.float64); U = _c(U, np.float64)
    n = 3 * NODES[etype]
    Ae = np.zeros((n, n)); be = np.zeros(n); Ne = np.zeros((n, n)); Nb = np.zeros(n); en = ctypes.c_double()
    rc = lib().oracle_nh_element(etype, _ptr(prm), _ptr(X), _ptr(U), _ptr(Ae), _ptr(be), _ptr(Ne), _ptr(Nb),
                                 ctypes.byref(en))
    if rc:
        raise InvertedElement(-1)
    return dict(A=Ae, b=be, NA=Ne, Nb=Nb, energy=en.value)


def nh_assemble(mesh, U, pat=None, **kw):
    """Jacobian and internal force of the whole mesh (3 dofs per node), element-index order.

    U: [n_nodes, 3].  Returns dict(row_ptr, col_idx, node_map, A, b, NA, Nb, energy).
    """
    if pat is None:
        pat = pattern(mesh, 3)
    rps, cols, nmap = pat
    prm = nh_params(**kw)
    E = mesh.n_elems
    A = np.zeros(cols.shape[0]); NA = np.zeros_like(A)
    b = np.zeros(mesh.n_nodes * 3); Nb = np.zeros_like(b)
    en = ctypes.c_double()
    types = _c(mesh.types, np.uint8); off = _c(mesh.conn_offsets, np.int64); conn = _c(mesh.conn, np.int32)
    coords = _c(mesh.coords, np.float64); U = _c(U, np.float64)
    rc = lib().oracle_nh_assemble(mesh.n_nodes, E, _ptr(types), _ptr(off), _ptr(conn), _ptr(coords), _ptr(prm),
                                  _ptr(U), _ptr(rps), _ptr(nmap), _ptr(A), _ptr(b), _ptr(NA), _ptr(Nb),
                                  ctypes.byref(en))
    if rc < 0:
        raise InvertedElement((-rc - 1) % E)
    return dict(row_ptr=rps, col_idx=cols, node_map=nmap, A=A, b=b, NA=NA, Nb=Nb, energy=en.value)
