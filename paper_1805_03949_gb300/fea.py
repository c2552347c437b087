"""Thin ctypes binding of the engine's C-ABI (``include/fea_gb300.h``).

The functions below carry the C names and only marshal arguments: every step
of the assembly runs in the CUDA kernels of ``libfea_gb300.so``.  Device
buffers are torch CUDA tensors owned by the caller; streams are torch streams
(the current stream by default).  There is no CPU fallback: importing this
module raises if the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libfea_gb300.so")

FEA_OK = 0
FEA_ERR_ARG = -1
FEA_ERR_OOM = -2
FEA_ERR_CUDA = -3
FEA_ERR_INVERTED_ELEMENT = -4
FEA_ERR_NO_CONVERGENCE = -5
FEA_ERR_TIMEOUT = -6
FEA_ERR_INDEX_OVERFLOW = -7
FEA_ERR_UNSUPPORTED = -8

FEA_TET4, FEA_PYR5, FEA_PRISM6, FEA_HEX8 = 0, 1, 2, 3
FEA_OP_DIFFUSION, FEA_OP_ELASTICITY, FEA_OP_J2, FEA_OP_NEOHOOKE = 0, 1, 2, 3
FEA_SCHED_PER_TYPE, FEA_SCHED_STEAL, FEA_SCHED_QUEUES, FEA_SCHED_QUEUES_STEAL = 0, 1, 2, 3
FEA_FP64, FEA_FP32_INTEGRATE, FEA_FP32_ADAPTIVE = 0, 1, 2
FEA_SCATTER_ATOMIC, FEA_SCATTER_COLOR, FEA_SCATTER_BLOCK, FEA_SCATTER_ROWS, FEA_SCATTER_MULTIDEP = 0, 1, 2, 3, 4


class FeaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class fea_mesh_desc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_elems", ctypes.c_int64),
                ("coords", ctypes.c_void_p), ("types", ctypes.c_void_p),
                ("conn_offsets", ctypes.c_void_p), ("conn", ctypes.c_void_p),
                ("on_device", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class fea_tuning(ctypes.Structure):
    _fields_ = [("block_elems", ctypes.c_int32), ("producer_warps", ctypes.c_int32),
                ("rows_block_nodes", ctypes.c_int32), ("chunk", ctypes.c_int32), ("ms", ctypes.c_float),
                ("candidates", ctypes.c_int32)]


class fea_batch_entry(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_void_p), ("row_ptr_d", ctypes.c_void_p), ("node_map_d", ctypes.c_void_p),
                ("A_d", ctypes.c_void_p), ("b_d", ctypes.c_void_p)]


class fea_operator(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("precision", ctypes.c_int32), ("scatter", ctypes.c_int32),
                ("tet_rule", ctypes.c_int32), ("k0", ctypes.c_double), ("k2", ctypes.c_double),
                ("source", ctypes.c_double), ("young", ctypes.c_double), ("poisson", ctypes.c_double),
                ("body_force", ctypes.c_double * 3), ("events", ctypes.POINTER(ctypes.c_void_p)),
                ("n_events", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("chunk", ctypes.c_int32), ("n_ctas", ctypes.c_int32),
                ("reserved2", ctypes.c_int32), ("queue_d", ctypes.c_void_p), ("queue_off_d", ctypes.c_void_p),
                ("item_ns_d", ctypes.c_void_p), ("item_cta_d", ctypes.c_void_p),
                ("sigma0", ctypes.c_double), ("sigma_inf", ctypes.c_double), ("delta", ctypes.c_double),
                ("hardening", ctypes.c_double), ("tol_g", ctypes.c_double), ("tol_step", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("reserved3", ctypes.c_int32),
                ("u_d", ctypes.c_void_p), ("state_in_d", ctypes.c_void_p), ("state_out_d", ctypes.c_void_p),
                ("yield_out_d", ctypes.c_void_p), ("iters_out_d", ctypes.c_void_p),
                ("lock_timeout_us", ctypes.c_int32), ("reserved4", ctypes.c_int32), ("span_d", ctypes.c_void_p),
                ("mass", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"engine library {LIB_PATH} is not built; run paper_1805_03949_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    sig = {
        "fea_last_error": (ctypes.c_char_p, []),
        "fea_abi_version": (I32, []),
        "fea_mesh_upload": (I32, [ctypes.POINTER(fea_mesh_desc), P, ctypes.POINTER(P)]),
        "fea_mesh_destroy": (I32, [P]),
        "fea_mesh_set_coords": (I32, [P, P, I32, P]),
        "fea_mesh_info": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "fea_pattern_size": (I32, [P, I32, ctypes.POINTER(I64), P]),
        "fea_build_csr_pattern": (I32, [P, I32, P, P, P, P]),
        "fea_assemble": (I32, [ctypes.POINTER(fea_operator), P, P, P, P, P, P]),
        "fea_check": (I32, [P, P]),
        "fea_assemble_launches": (I32, [ctypes.POINTER(fea_operator), P, ctypes.POINTER(I32)]),
        "fea_row_ptr_from_counts_noalloc": (I32, [P, I64, P, P]),
        "fea_work_items": (I32, [P, I32, ctypes.POINTER(I64), P, P, P]),
        "fea_costmodel_create": (I32, [I32, P, ctypes.POINTER(P)]),
        "fea_costmodel_destroy": (I32, [P]),
        "fea_costmodel_get_params": (I32, [P, P, P]),
        "fea_costmodel_fit_scaler": (I32, [P, P, P, I64, P]),
        "fea_costmodel_grad": (I32, [P, P, P, I64, P, P, P]),
        "fea_costmodel_train": (I32, [P, P, P, I64, I32, ctypes.c_float, P, P]),
        "fea_costmodel_predict": (I32, [P, P, I64, P, P]),
        "fea_item_features": (I32, [P, I32, P, P, P, P]),
        "fea_pack_lpt": (I32, [P, I64, I32, P, P, P]),
        "fea_element_loop": (I32, [ctypes.POINTER(fea_operator), P, P, P]),
        "fea_spmv": (I32, [P, I32, P, P, P, P, P, P, P]),
        "fea_element_loop_grid": (I32, [ctypes.POINTER(fea_operator), P, ctypes.POINTER(I32)]),
        "fea_batch_create": (I32, [ctypes.POINTER(fea_operator), I32, P, ctypes.POINTER(P)]),
        "fea_batch_destroy": (I32, [P]),
        "fea_batch_set_config": (I32, [P, I32, I32]),
        "fea_batch_info": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "fea_batch_autotune": (I32, [P, I32, P, ctypes.POINTER(I32), ctypes.POINTER(I32),
                                     ctypes.POINTER(ctypes.c_float)]),
        "fea_batch_capture": (I32, [P, P]),
        "fea_batch_assemble": (I32, [P, P]),
        "fea_batch_latency": (I32, [P, P, P]),
        "fea_persistent_grid": (I32, [ctypes.POINTER(fea_operator), P, ctypes.POINTER(I32)]),
        "fea_mesh_set_rows_block": (I32, [P, I32]),
        "fea_rows_plan_info": (I32, [P, ctypes.POINTER(I64)]),
        "fea_color_info": (I32, [P, P, ctypes.POINTER(I32)]),
        "fea_mesh_set_block_elems": (I32, [P, I32]),
        "fea_multidep_plan": (I32, [P, I32, ctypes.POINTER(I64), P, P, P, P]),
        "fea_multidep_hold": (I32, [P, I32, I32]),
        "fea_peak_probe": (I32, [I32, I64, ctypes.POINTER(ctypes.c_double), P]),
        "fea_convert": (I32, [I32, P, P, I64, P]),
        "fea_mesh_set_pipe_split": (I32, [P, I32]),
        "fea_autotune": (I32, [ctypes.POINTER(fea_operator), P, P, P, P, P, I32, P, ctypes.POINTER(fea_tuning)]),
    }
    for name, (rt, at) in sig.items():
        f = getattr(lib, name)
        f.restype = rt
        f.argtypes = at
    return lib


_lib = _load()


def lib():
    """The loaded engine library (ctypes.CDLL)."""
    return _lib


def _check(rc: int):
    if rc != FEA_OK:
        raise FeaError(rc, _lib.fea_last_error().decode())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, dtype=None, min_numel=None, name="tensor") -> ctypes.c_void_p:
    """Device pointer of a contiguous CUDA tensor on the current device (None passes NULL).

    dtype and min_numel, where given, are checked too: the library reads the
    pointer as that element type and writes up to min_numel elements."""
    if t is None:
        return ctypes.c_void_p(None)
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise TypeError(f"{name}: expected a contiguous CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on {t.device}, but the current device is cuda:{torch.cuda.current_device()}")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name}: needs at least {min_numel} elements, has {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def fea_last_error() -> str:
    """Message of the last failing call on this thread."""
    return _lib.fea_last_error().decode()


def fea_abi_version() -> int:
    """ABI version of the loaded library."""
    return int(_lib.fea_abi_version())


def fea_mesh_upload(coords, types, conn_offsets, conn, stream=None) -> ctypes.c_void_p:
    """Upload a mesh (numpy host arrays or contiguous CUDA tensors); returns the handle."""
    on_device = isinstance(coords, torch.Tensor) and coords.is_cuda
    keep = []
    if on_device:
        arrs = [coords.to(torch.float64).contiguous(), types.to(torch.uint8).contiguous(),
                conn_offsets.to(torch.int64).contiguous(), conn.to(torch.int32).contiguous()]
        ptrs = [a.data_ptr() for a in arrs]
        keep = arrs
    else:
        arrs = [np.ascontiguousarray(coords, dtype=np.float64), np.ascontiguousarray(types, dtype=np.uint8),
                np.ascontiguousarray(conn_offsets, dtype=np.int64), np.ascontiguousarray(conn, dtype=np.int32)]
        ptrs = [a.ctypes.data for a in arrs]
        keep = arrs
    d = fea_mesh_desc(n_nodes=int(arrs[0].shape[0]), n_elems=int(arrs[1].shape[0]), coords=ptrs[0],
                      types=ptrs[1], conn_offsets=ptrs[2], conn=ptrs[3], on_device=1 if on_device else 0)
    h = ctypes.c_void_p()
    _check(_lib.fea_mesh_upload(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
    del keep
    return h


def fea_mesh_set_coords(h, coords, stream=None):
    """New node coordinates: a contiguous float64 CUDA tensor, or a numpy array / CPU tensor."""
    if isinstance(coords, torch.Tensor) and coords.is_cuda:
        _check(_lib.fea_mesh_set_coords(h, _dptr(coords), 1, _stream(stream)))
    else:
        if isinstance(coords, torch.Tensor):
            arr = coords.contiguous()
            ptr = arr.data_ptr()
        else:
            arr = np.ascontiguousarray(coords, dtype=np.float64)
            ptr = arr.ctypes.data
        _check(_lib.fea_mesh_set_coords(h, ctypes.c_void_p(ptr), 0, _stream(stream)))


def fea_mesh_destroy(h):
    """Free a mesh handle and its device buffers."""
    _check(_lib.fea_mesh_destroy(h))


def fea_mesh_info(h):
    """(n_nodes, n_elems, map_len), map_len = sum of n_e^2 over the elements."""
    n, e, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.fea_mesh_info(h, ctypes.byref(n), ctypes.byref(e), ctypes.byref(m)))
    return n.value, e.value, m.value


def fea_pattern_size(h, ndof: int, stream=None) -> int:
    """Build the node graph and return the scalar nonzero count for ndof (1 or 3) dofs per node."""
    nnz = ctypes.c_int64()
    _check(_lib.fea_pattern_size(h, ndof, ctypes.byref(nnz), _stream(stream)))
    return nnz.value


def fea_build_csr_pattern(h, ndof: int, row_ptr, col_idx, node_map, stream=None):
    """Write row_ptr (int64), col_idx (int32, or None) and node_map (int32, or None) CUDA tensors."""
    n, _, mlen = fea_mesh_info(h)
    _check(_lib.fea_build_csr_pattern(h, ndof, _dptr(row_ptr, torch.int64, n * ndof + 1, "row_ptr"),
                                      _dptr(col_idx, torch.int32, name="col_idx"),
                                      _dptr(node_map, torch.int32, mlen, "node_map"), _stream(stream)))


def fea_assemble(op: "fea_operator", h, row_ptr, node_map, A, b, stream=None):
    """Overwrite A (float64 [nnz]) and b (float64 [n_nodes * ndof]) with the assembled system."""
    _check(_lib.fea_assemble(ctypes.byref(op), h, _dptr(row_ptr, torch.int64, name="row_ptr"),
                             _dptr(node_map, torch.int32, name="node_map"), _dptr(A, torch.float64, name="A"),
                             _dptr(b, torch.float64, name="b"), _stream(stream)))


def fea_check(h, stream=None):
    """Wait for the stream; raise FeaError if the mesh latched a device error."""
    _check(_lib.fea_check(h, _stream(stream)))


def fea_row_ptr_from_counts_noalloc(counts, row_ptr, stream=None):
    """Row pointers from int32 row lengths into ``row_ptr`` (n + 1 int64), no device allocation.

    For callers that cannot let the library allocate device memory; see the
    declaration in fea_gb300.h for the size limit and the shared scratch.
    """
    n = int(counts.numel())
    _check(_lib.fea_row_ptr_from_counts_noalloc(_dptr(counts, torch.int32, name="counts"), n,
                                                _dptr(row_ptr, torch.int64, n + 1, name="row_ptr"),
                                                _stream(stream)))


def fea_mesh_set_rows_block(h, block_nodes: int):
    """Nodes per CTA block of the owner-computes rows scatter (1..512)."""
    _check(_lib.fea_mesh_set_rows_block(h, int(block_nodes)))


def fea_mesh_set_block_elems(h, block_elems: int):
    """Elements per block of the block-task scatter."""
    _check(_lib.fea_mesh_set_block_elems(h, int(block_elems)))


def fea_mesh_set_pipe_split(h, producer_warps: int):
    """Producer warps (4..8 of 16) of the pipelined block-task kernel."""
    _check(_lib.fea_mesh_set_pipe_split(h, int(producer_warps)))


def fea_autotune(op: "fea_operator", h, row_ptr, node_map, A, b, reps: int = 5, stream=None) -> dict:
    """Time the candidate launch parameters of op's path on the mesh, keep the fastest (see the header)."""
    t = fea_tuning()
    _check(_lib.fea_autotune(ctypes.byref(op), h, _dptr(row_ptr, torch.int64, name="row_ptr"),
                             _dptr(node_map, torch.int32, name="node_map"), _dptr(A, torch.float64, name="A"),
                             _dptr(b, torch.float64, name="b"), int(reps), _stream(stream), ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in fea_tuning._fields_}


def autotune(op: "fea_operator", system: "System", key: str, cache: str | None = None, reps: int = 5) -> dict:
    """fea_autotune with a JSON cache: the choice for `key` (a name for the mesh
    and operator) is read from `cache` if present and applied without timing;
    otherwise it is timed and written there."""
    import json
    entries = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            entries = json.load(f)
    if key in entries:
        c = entries[key]
        fea_mesh_set_block_elems(system.handle, c["block_elems"])
        fea_mesh_set_pipe_split(system.handle, c["producer_warps"])
        fea_mesh_set_rows_block(system.handle, c["rows_block_nodes"])
        op.chunk = c["chunk"]
        return dict(c, cached=True)
    c = fea_autotune(op, system.handle, system.row_ptr, system.node_map, system.A, system.b, reps)
    if cache:
        entries[key] = c
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(entries, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return dict(c, cached=False)


def fea_rows_plan_info(h) -> dict:
    """Statistics of the mesh's current owner-computes rows plan (zeros if none)."""
    arr = (ctypes.c_int64 * 8)()
    _check(_lib.fea_rows_plan_info(h, arr))
    keys = ["blocks", "block_nodes", "max_local", "max_halo", "tasks", "contributions", "halo_elements", "bytes"]
    return dict(zip(keys, list(arr)))


def fea_color_info(h, n_elems: int):
    """(n_colors, int32 numpy array of every element's color class)."""
    n = ctypes.c_int()
    colors = np.zeros(n_elems, dtype=np.int32)
    _check(_lib.fea_color_info(h, ctypes.c_void_p(colors.ctypes.data), ctypes.byref(n)))
    return n.value, colors


def fea_multidep_plan(h, chunk: int, n_elems: int) -> dict:
    """The FEA_SCATTER_MULTIDEP plan of `chunk` (built if needed): counts,
    neighbour lists (CSR), priority order and local colors (numpy)."""
    info = (ctypes.c_int64 * 4)()
    _check(_lib.fea_multidep_plan(h, int(chunk), info, None, None, None, None))
    n_sub, n_nb = int(info[0]), int(info[1])
    nb_off = np.zeros(n_sub + 1, dtype=np.int64)
    nb = np.zeros(max(n_nb, 1), dtype=np.int32)
    order = np.zeros(max(n_sub, 1), dtype=np.int32)
    color = np.zeros(max(n_elems, 1), dtype=np.int32)
    _check(_lib.fea_multidep_plan(h, int(chunk), info, ctypes.c_void_p(nb_off.ctypes.data),
                                  ctypes.c_void_p(nb.ctypes.data), ctypes.c_void_p(order.ctypes.data),
                                  ctypes.c_void_p(color.ctypes.data)))
    return {"subdomains": n_sub, "entries": n_nb, "max_neighbours": int(info[2]), "max_colors": int(info[3]),
            "nb_off": nb_off, "nb": nb[:n_nb], "order": order[:n_sub], "color": color[:n_elems]}


def fea_multidep_hold(h, subdomain: int, held: bool):
    """Hold or free one subdomain's lock in every later multidependence launch (tests of the bounded wait)."""
    _check(_lib.fea_multidep_hold(h, int(subdomain), 1 if held else 0))


def fea_work_items(h, chunk: int = 0):
    """Work items of the persistent schedules: (type, first, count) int32 arrays."""
    n = ctypes.c_int64()
    _check(_lib.fea_work_items(h, chunk, ctypes.byref(n), None, None, None))
    t = np.zeros(n.value, dtype=np.int32); f = np.zeros_like(t); c = np.zeros_like(t)
    _check(_lib.fea_work_items(h, chunk, ctypes.byref(n), t.ctypes.data_as(ctypes.c_void_p),
                               f.ctypes.data_as(ctypes.c_void_p), c.ctypes.data_as(ctypes.c_void_p)))
    return t, f, c


def fea_persistent_grid(op: "fea_operator", h) -> int:
    """CTAs of the persistent launch of op on the mesh (the queue count for packed schedules)."""
    n = ctypes.c_int32()
    _check(_lib.fea_persistent_grid(ctypes.byref(op), h, ctypes.byref(n)))
    return int(n.value)


# ---------------------------------------------------------------------------
# learned cost model and queue packing (costmodel.cu)
# ---------------------------------------------------------------------------

def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def fea_costmodel_create(n_in: int, params) -> ctypes.c_void_p:
    """New cost model with n_in features (1..8) and initial float32 parameters."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    h = ctypes.c_void_p()
    _check(_lib.fea_costmodel_create(n_in, _np_ptr(p), ctypes.byref(h)))
    return h


def fea_costmodel_destroy(h):
    """Free a cost model."""
    _check(_lib.fea_costmodel_destroy(h))


def fea_costmodel_get_params(h, n_in: int):
    """(parameters, scaler) as float32 numpy arrays."""
    n = 32 * n_in + 32 + 32 * 32 + 32 + 32 + 1
    p = np.zeros(n, dtype=np.float32); sc = np.zeros(2 * n_in + 2, dtype=np.float32)
    _check(_lib.fea_costmodel_get_params(h, _np_ptr(p), _np_ptr(sc)))
    return p, sc


def fea_costmodel_fit_scaler(h, X, y, stream=None):
    """Fit the feature and target standardisation to X [n, n_in] and y [n] (float32 CUDA)."""
    _check(_lib.fea_costmodel_fit_scaler(h, _dptr(X), _dptr(y), X.shape[0], _stream(stream)))


def fea_costmodel_grad(h, X, y, n_params: int, stream=None):
    """(gradient [n_params], loss [1]) at the current parameters, as float32 CUDA tensors."""
    g = torch.empty(n_params, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(_lib.fea_costmodel_grad(h, _dptr(X), _dptr(y), X.shape[0], _dptr(g), _dptr(loss), _stream(stream)))
    return g, loss


def fea_costmodel_train(h, X, y, epochs: int, lr: float, stream=None):
    """Full-batch Adam epochs; returns the last epoch's loss (float32 CUDA [1])."""
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(_lib.fea_costmodel_train(h, _dptr(X), _dptr(y), X.shape[0], epochs, lr, _dptr(loss), _stream(stream)))
    return loss


def fea_costmodel_predict(h, X, stream=None):
    """Predicted costs for X [n, n_in] (float32 CUDA [n], target units)."""
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _check(_lib.fea_costmodel_predict(h, _dptr(X), X.shape[0], _dptr(y), _stream(stream)))
    return y


def fea_item_features(h, chunk: int, n_items: int, u=None, state_in=None, device="cuda", stream=None):
    """Features of the work items of fea_work_items(h, chunk): float32 CUDA [n_items, 6]."""
    X = torch.empty((n_items, 6), dtype=torch.float32, device=device)
    _check(_lib.fea_item_features(h, chunk, _dptr(u),
                                  _dptr(state_in), _dptr(X), _stream(stream)))
    return X


def fea_pack_lpt(costs, n_queues: int):
    """Host LPT packing: (queue ids int32, offsets int64 [n_queues + 1], loads float64)."""
    c = np.ascontiguousarray(costs, dtype=np.float64)
    q = np.zeros(len(c), dtype=np.int32); off = np.zeros(n_queues + 1, dtype=np.int64)
    load = np.zeros(n_queues, dtype=np.float64)
    _check(_lib.fea_pack_lpt(_np_ptr(c), len(c), n_queues, _np_ptr(q), _np_ptr(off), _np_ptr(load)))
    return q, off, load


# ---------------------------------------------------------------------------
# batches of meshes (batch.cu)
# ---------------------------------------------------------------------------

class Batch:
    """Many Systems assembled by one persistent launch (optionally a CUDA graph)."""

    def __init__(self, op: "fea_operator", systems):
        self.systems = list(systems)
        arr = (fea_batch_entry * len(self.systems))()
        for k, s in enumerate(self.systems):
            arr[k].mesh = s.handle
            arr[k].row_ptr_d = s.row_ptr.data_ptr()
            arr[k].node_map_d = s.node_map.data_ptr()
            arr[k].A_d = s.A.data_ptr()
            arr[k].b_d = s.b.data_ptr()
        self.handle = ctypes.c_void_p()
        _check(_lib.fea_batch_create(ctypes.byref(op), len(self.systems), arr, ctypes.byref(self.handle)))

    def set_config(self, chunk: int, n_ctas: int):
        """Change the work-item size and the grid (drops a captured graph)."""
        _check(_lib.fea_batch_set_config(self.handle, chunk, n_ctas))

    def info(self):
        """Items, chunk size and grid of the current configuration."""
        n, c, g = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.fea_batch_info(self.handle, ctypes.byref(n), ctypes.byref(c), ctypes.byref(g)))
        return dict(items=n.value, chunk=c.value, grid=g.value)

    def autotune(self, reps: int = 3, stream=None):
        """Time chunk sizes and grids, keep the fastest; returns it."""
        c, g, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        _check(_lib.fea_batch_autotune(self.handle, reps, _stream(stream), ctypes.byref(c), ctypes.byref(g),
                                       ctypes.byref(ms)))
        return dict(chunk=c.value, grid=g.value, ms=ms.value)

    def capture(self, stream=None):
        """Capture one assembly as a CUDA graph; later assemble() calls replay it."""
        _check(_lib.fea_batch_capture(self.handle, _stream(stream)))

    def assemble(self, stream=None):
        """Assemble every system of the batch (overwrite)."""
        _check(_lib.fea_batch_assemble(self.handle, _stream(stream)))

    def latency_ns(self, stream=None):
        """Per-mesh latency of the last assembly, ns (uint64 numpy)."""
        out = np.zeros(len(self.systems), dtype=np.uint64)
        _check(_lib.fea_batch_latency(self.handle, out.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
        return out

    def close(self):
        """Destroy the batch handle."""
        if self.handle:
            _check(_lib.fea_batch_destroy(self.handle))
            self.handle = None


def fea_spmv(h, ndof: int, row_ptr, A, x, y, glob=None, shared=None, stream=None):
    """y = A x through the mesh's node graph; with glob/shared, add a subdomain's partial rows into a global y."""
    _check(_lib.fea_spmv(h, ndof, _dptr(row_ptr), _dptr(A), _dptr(x), _dptr(y), _dptr(glob), _dptr(shared),
                         _stream(stream)))


def fea_element_loop(op: "fea_operator", h, stress=None, stream=None):
    """The J2 Gauss-point update of every element, without a scatter (stress: float64 [n_elems, 8, 6] or None)."""
    _check(_lib.fea_element_loop(ctypes.byref(op), h, _dptr(stress), _stream(stream)))


def fea_element_loop_grid(op: "fea_operator", h) -> int:
    """CTAs of the persistent element loop of op on the mesh."""
    n = ctypes.c_int32()
    _check(_lib.fea_element_loop_grid(ctypes.byref(op), h, ctypes.byref(n)))
    return int(n.value)


def fea_peak_probe(kind: int, iters: int, stream=None) -> float:
    """Measured FMA rate of the current GPU in flop/s: kind 0 FP64, 1 FP32."""
    f = ctypes.c_double()
    _check(_lib.fea_peak_probe(int(kind), int(iters), ctypes.byref(f), _stream(stream)))
    return f.value


def fea_convert(x: "torch.Tensor", stream=None) -> "torch.Tensor":
    """The kernels' precision conversion of a CUDA tensor: float32 -> float64
    (exact widening) or float64 -> float32 (round to nearest even)."""
    if not isinstance(x, torch.Tensor) or x.dtype not in (torch.float32, torch.float64):
        raise TypeError("fea_convert: a float32 or float64 CUDA tensor")
    d = 0 if x.dtype == torch.float32 else 1
    out = torch.empty(x.shape, dtype=torch.float64 if d == 0 else torch.float32, device=x.device)
    _check(_lib.fea_convert(d, _dptr(x, x.dtype, name="x"), _dptr(out, out.dtype, x.numel(), "out"), x.numel(),
                            _stream(stream)))
    return out


def fea_assemble_launches(op: "fea_operator", h) -> int:
    """Kernels one fea_assemble call with op launches on the mesh."""
    n = ctypes.c_int()
    _check(_lib.fea_assemble_launches(ctypes.byref(op), h, ctypes.byref(n)))
    return n.value


def set_events(op: "fea_operator", events) -> None:
    """Attach torch.cuda.Event objects (already recorded once, so they exist) as the profiling hook."""
    if not events:
        op.events = None
        op.n_events = 0
        return
    arr = (ctypes.c_void_p * len(events))(*[e.cuda_event for e in events])
    op._event_array = arr
    op.events = ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p))
    op.n_events = len(events)


# ---------------------------------------------------------------------------
# convenience: operator construction and a mesh + pattern + buffers bundle
# ---------------------------------------------------------------------------

def make_operator(kind=FEA_OP_DIFFUSION, precision=FEA_FP64, scatter=FEA_SCATTER_ATOMIC, tet_rule=1,
                  k0=1.0, k2=0.0, source=1.0, young=1.0, poisson=0.3, body_force=(1.0, 1.0, 1.0),
                  schedule=FEA_SCHED_PER_TYPE, chunk=0, n_ctas=0, queue=None, queue_off=None, item_ns=None,
                  item_cta=None, sigma0=1e-3, sigma_inf=3e-3, delta=300.0, hardening=1e-2, tol_g=1e-13,
                  tol_step=1e-15, max_iter=12, u=None, state_in=None, state_out=None, yield_out=None,
                  iters_out=None, lock_timeout_us=0, span=None, mass=0.0) -> fea_operator:
    """Operator struct; tensors (device) are referenced by pointer, the caller keeps them alive."""
    op = fea_operator()
    op.kind, op.precision, op.scatter, op.tet_rule = kind, precision, scatter, tet_rule
    op.k0, op.k2, op.source = k0, k2, source
    op.young, op.poisson = young, poisson
    for c in range(3):
        op.body_force[c] = body_force[c]
    op.schedule, op.chunk, op.n_ctas = schedule, chunk, n_ctas
    op.queue_d, op.queue_off_d = _dptr(queue), _dptr(queue_off)
    op.item_ns_d, op.item_cta_d = _dptr(item_ns), _dptr(item_cta)
    op.sigma0, op.sigma_inf, op.delta, op.hardening = sigma0, sigma_inf, delta, hardening
    op.tol_g, op.tol_step, op.max_iter = tol_g, tol_step, max_iter
    op.u_d, op.state_in_d, op.state_out_d = _dptr(u), _dptr(state_in), _dptr(state_out)
    op.yield_out_d, op.iters_out_d = _dptr(yield_out), _dptr(iters_out)
    op.lock_timeout_us, op.span_d = lock_timeout_us, _dptr(span)
    op.mass = mass
    return op


@dataclass
class System:
    """A mesh handle with its CSR pattern, map and value buffers on one device."""

    handle: ctypes.c_void_p
    ndof: int
    n_nodes: int
    n_elems: int
    row_ptr: torch.Tensor
    col_idx: torch.Tensor
    node_map: torch.Tensor
    A: torch.Tensor
    b: torch.Tensor
    extra: dict = field(default_factory=dict)

    @classmethod
    def from_mesh(cls, mesh, ndof: int, device="cuda", stream=None, with_cols: bool = True) -> "System":
        h = fea_mesh_upload(mesh.coords, mesh.types, mesh.conn_offsets, mesh.conn, stream)
        n, e, mlen = fea_mesh_info(h)
        nnz = fea_pattern_size(h, ndof, stream)
        rp = torch.empty(n * ndof + 1, dtype=torch.int64, device=device)
        col = torch.empty(nnz if with_cols else 0, dtype=torch.int32, device=device)
        nmap = torch.empty(mlen, dtype=torch.int32, device=device)
        fea_build_csr_pattern(h, ndof, rp, col if with_cols else None, nmap, stream)
        A = torch.empty(nnz, dtype=torch.float64, device=device)
        b = torch.empty(n * ndof, dtype=torch.float64, device=device)
        return cls(h, ndof, n, e, rp, col, nmap, A, b)

    def assemble(self, op: fea_operator, stream=None):
        fea_assemble(op, self.handle, self.row_ptr, self.node_map, self.A, self.b, stream)

    def check(self, stream=None):
        fea_check(self.handle, stream)

    def close(self):
        if self.handle is not None:
            fea_mesh_destroy(self.handle)
            self.handle = None
