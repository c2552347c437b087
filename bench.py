"""Benchmark of the finite element assembly engine on one GB300 (one rank per GPU).

Workload (default): 3D linear elasticity on hex8, a 128^3 unit cube with
interior nodes jittered by U(-0.2h, 0.2h) (PCG64 seed 2): 2,097,152 elements,
2,146,689 nodes, 513,599,625 scalar nonzeros, 2x2x2 Gauss.  This is the
synthetic stand-in for the paper's large mechanics meshes (the Iter and
respiratory meshes, Sec. 2.1.5 / 2.2.2, are not available).

One step = one ``fea_assemble`` call (zero A and b, integrate every element,
scatter into the CSR system) on a mesh, pattern and map already resident in
HBM.  The metric is assembled elements per second; the comparator is the
plain per-type FP64 atomic assembly on the same GPU in the same run.  A (4.1
GB) is far larger than L2 (129 MB), so no L2 flush is needed between steps.

Under torchrun each rank assembles its own copy of the workload (the
partial-row decomposition of Sec. 3.1 needs no communication during
assembly): weak scaling, value = all ranks' elements / max rank time.

``--impl reference`` times the CPU oracle (single thread, element-index
order) on a bounded slab of the same mesh and prints the same line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_FP64_TFLOPS = 1.25     # GB300 FP64, NVIDIA's nominal dense rate
NOMINAL_FP32_TFLOPS = 80.5     # 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz

METRIC = "assembled elements/s and % roofline vs plain atomic FP64 assembly, same GB300"

# DRAM bytes (read + write) of one launch of a kernel at the 128^3 workload: an
# ncu capture of the 64^3 case in the same configuration (inputs larger than
# L2), scaled by the element count, which the traffic grows with.  Keyed by
# (kernel, elements per block, producer warps) for the block-task kernel, whose
# traffic depends on its configuration; remove an entry whenever its kernel
# changes, and a configuration without an entry reports no traffic.
TRAFFIC_BYTES = {("k_block_pipe", 64, 6): 8.0 * (394735616 + 557147648)}

# the kernel each variant spends its step in
DOMINANT_KERNEL = {"atomic": "k_assemble_tile", "color": "k_assemble_tile (one launch per color)",
                   "rows": "k_rows_assemble", "block": "k_block_pipe (block-task plan, geometry fused)"}


def _peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def measured_peaks(fea):
    """Roofline denominators: HBM copy bandwidth (MEASURED_PEAKS.json) and the FP64 and
    FP32 FMA rates measured on this GPU by the engine's probe (nominal where it fails)."""
    hbm, kind = _peaks()
    out = {"hbm": hbm * 1e9, "hbm_source": kind,
           "fp64_nominal": NOMINAL_FP64_TFLOPS * 1e12, "fp32_nominal": NOMINAL_FP32_TFLOPS * 1e12}
    for key, k, iters in (("fp64", 0, 20000), ("fp32", 1, 1000000)):
        try:
            out[key] = fea.fea_peak_probe(k, iters)
            out[key + "_source"] = "measured (fea_peak_probe: FMA chains on every SM, CUDA events)"
        except Exception as e:  # noqa: BLE001 -- report the nominal rate instead
            out[key] = out[key + "_nominal"]
            out[key + "_source"] = f"nominal (probe failed: {e})"
    return out


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, out_dir: str):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload and algorithmic counts
# ---------------------------------------------------------------------------

# The assembly variants of the headline workload: name -> (fea_precision,
# fea_scatter suffix).  "fp32a" is FP32 geometry with the FP64 redo of
# distorted elements only (kappa_F(J) > 12); the multidependence variant runs
# subdomains of 128 elements under neighbour-set locks.
VARIANTS = {
    "fp64_atomic": (0, "ATOMIC"),
    "fp32_atomic": (1, "ATOMIC"),
    "fp32_rows": (1, "ROWS"),
    "fp64_rows": (0, "ROWS"),
    "fp32_color": (1, "COLOR"),
    "fp32_block": (1, "BLOCK"),
    "fp32_multidep": (1, "MULTIDEP"),
    "fp32a_atomic": (2, "ATOMIC"),
    "fp32a_rows": (2, "ROWS"),
}


# variants whose launch parameters the autotuner picks before they are timed
TUNED_VARIANTS = ("fp32_block", "fp32_rows", "fp32_multidep")


def variant_operators(fea) -> dict:
    """Linear elasticity (E = 1, nu = 0.3) operators of the variants, in table order."""
    return {name: fea.make_operator(kind=fea.FEA_OP_ELASTICITY, precision=prec,
                                    scatter=getattr(fea, "FEA_SCATTER_" + sc), poisson=0.3)
            for name, (prec, sc) in VARIANTS.items()}


def hex_cube_mesh(n=128):
    """The headline workload's mesh: n^3 hex8 cube, interior nodes jittered by +-0.2h (PCG64 seed 2)."""
    from paper_1805_03949_gb300 import meshgen as mg
    return mg.hex_cube(n, 0.2, 2)


def algorithmic_bytes(n_nodes, n_elems, nnz, nn=8, ndof=3):
    """Bytes one assembly must move: A and b written once, inputs read once.

    per element: conn 4*nn, node_map 4*nn^2; per node: coords 24, row_ptr 8*ndof,
    b 8*ndof; per nonzero: A 8.
    """
    return 8 * nnz + n_nodes * (24 + 8 * ndof + 8 * ndof) + n_elems * (4 * nn + 4 * nn * nn)


def algorithmic_bytes_spmv(n_nodes, nnz, ndof=3):
    """Bytes of y = A x read through the node graph: A once, one int32 node
    column per node-level nonzero, the node row starts, the scalar row starts,
    x read once and y written once."""
    nnz_node = nnz // (ndof * ndof)
    return (8 * nnz + 4 * nnz_node + 8 * (n_nodes + 1) + 8 * (ndof * n_nodes + 1)
            + 8 * ndof * n_nodes + 8 * ndof * n_nodes)


def algorithmic_flops_hex_elasticity(n_elems, n_nodes, nnz, nq=8, nn=8):
    """FP32 and FP64 arithmetic of one FP32-integrate hex8 elasticity assembly (FMA = 2 flop).

    FP64 geometry (per element): modal transform of the corners 3 stages x 8 x 3
    adds; the Jacobian's column c depends only on the other two coordinates
    of the Gauss point, so it takes 4 distinct values over the 8 points: 3
    columns x 4 values x 9 FMA per element; per point: cofactors 9 mul + 9
    FMA, det 1 mul + 2 FMA, w det J 2 mul.
    FP64 accumulation: the contributions to one entry are FP32 and are summed
    in FP64, so an entry with k contributions takes at least k - 1 FP64 adds.
    A is symmetric, so only the (a <= b) blocks of every element count: 36 x 9
    contributions per element into the (nnz + 9 n_nodes) / 2 entries of the
    upper blocks; b: 8 x 3 contributions per element into 3 n_nodes entries.
    FP32 (per point): scaled gradients 8 x 9 FMA + 24 mul, scale 3; per (a <= b)
    block the moment g_a g_b^T, 9 FMA; RHS 3 FMA per (a, point); once per block
    lam M + mu M^T + mu tr(M) I, 33.
    """
    geometry = 72 + 2 * 108 + nq * ((9 + 2 * 9) + (1 + 2 * 2) + 2)
    blocks = nn * (nn + 1) // 2
    accumulate = (blocks * 9 * n_elems - (nnz + 9 * n_nodes) // 2) + (3 * nn * n_elems - 3 * n_nodes)
    fp32 = nq * ((2 * 72 + 24 + 3) + blocks * 2 * 9 + nn * 2 * 3) + blocks * 33
    return {"fp64": n_elems * geometry + accumulate, "fp64_geometry": n_elems * geometry,
            "fp64_accumulate": accumulate, "fp32": n_elems * fp32}


# ---------------------------------------------------------------------------
# algorithmic work of any workload: per element type, operator and precision
# ---------------------------------------------------------------------------

NODES_PER_TYPE = {0: 4, 1: 5, 2: 6, 3: 8}
TYPE_NAMES = {0: "tet4", 1: "pyr5", 2: "prism6", 3: "hex8"}
OP_DIFFUSION, OP_ELASTICITY, OP_J2 = 0, 1, 2


def element_flops(etype, op, nq, k_varies=False):
    """Arithmetic of one element (FMA = 2 flop, div / sqrt / exp = 1), split by role.

    geometry (FP64 in every precision): the Jacobian J, its cofactors C
      (9 mul + 9 FMA), det J (1 mul + 2 FMA) and w det J per point.
      hex8 (2x2x2 rule, modal form): 3 stages x 8 corners x 3 adds of the
        Walsh-Hadamard transform of the corners; J from 4 modal coefficients
        per entry (3 FMA), column c at the 4 distinct pairs of the other two
        point coordinates (3 x 4 x 9 FMA per element); w det J (2 mul) per
        point;
      tet4 (affine): 3 x 3 edge differences, C, det and 1/det once; w det J
        (1 mul) per point;
      pyr5, prism6: 3 (nn - 1) differences to node 0 once; per point J = sum
        over the other nodes (9 (nn - 1) FMA), C, det, w det J (1 mul).
    coords (FP64, diffusion with k = k0 + k2 x^2 only): x_q = sum_a N_a x_a,
      nn FMA per point.
    grad: the scaled gradients g_a = s C grad_xi N_a, 9 FMA + 3 mul per node
      and 3 for s = sqrt(w det J) / det J, per point; an affine tet's gradients
      are constant, taken once with s = 1 / det J from its geometry.
    prod: diffusion, per point k_q g_a (3 mul per node) and, per (a <= b)
      pair, 3 FMA accumulating k_q g_a . g_b into A_ab, plus k_q = k0 + k2 x_q^2
      (mul + FMA) where k varies; elasticity, per point and (a <= b) block the
      moment M_ab += g_a g_b^T (9 FMA), and once per block lam M + mu M^T +
      mu tr(M) I (2 adds and 1 mul for the trace, 9 x (mul + FMA), 3 adds).
      An affine tet, whose gradients are constant, takes its products once:
      the weight sum W = sum_q w_q det J k_q (1 FMA per point, and k_q), then
      per pair a dot product (3 FMA) times W (1 mul) for diffusion; for
      elasticity lam W and mu W (2 mul) and per block M (9 FMA) and the
      combination (33).  J2 (op 2): per point and block three moment sums
      weighted by lam', mu' and beta (27 FMA), per node and point lam' g_a,
      mu' g_a (6 mul), h_a = n g_a (9 FMA), beta h_a (3 mul) and the internal
      force sigma g_a (9 FMA), and per block their combination (23 adds).
    rhs: w det J f_c N_a, 1 FMA per node, component and point.
    """
    nn = NODES_PER_TYPE[etype]
    pairs = nn * (nn + 1) // 2
    d = 1 if op == OP_DIFFUSION else 3
    affine = etype == 0
    if etype == 3:
        geometry = 72 + 2 * 108 + nq * (27 + 5 + 2)
    elif affine:
        geometry = 9 + 27 + 5 + 1 + nq
    else:
        geometry = 3 * (nn - 1) + nq * (2 * 9 * (nn - 1) + 27 + 5 + 1)
    coords = nq * 2 * nn if (op == OP_DIFFUSION and k_varies) else 0
    grad = 21 * nn if affine else nq * (21 * nn + 3)
    kq = 3 if k_varies else 0
    if op == OP_DIFFUSION:
        prod = 7 * pairs + nq * (2 + kq) if affine else nq * (kq + 3 * nn + 6 * pairs)
    elif op == OP_J2:
        # three weighted moment sums per (a <= b) block and point (27 FMA); per
        # node and point lam' g_a, mu' g_a (6 mul), h_a = n g_a (9 FMA), beta
        # h_a (3 mul) and the internal force sigma g_a (9 FMA); once per block
        # the combination (23 adds)
        prod = nq * (54 * pairs + 45 * nn) + 23 * pairs
    else:
        # M_ab = sum_q g_a g_b^T (9 FMA per block and point), then once per
        # block lam M + mu M^T + mu tr(M) I (33); an affine tet forms M once,
        # with lam W and mu W (2 mul) and W = sum_q w_q det J (1 FMA per point)
        prod = 51 * pairs + 2 + 2 * nq if affine else nq * 18 * pairs + 33 * pairs
    rhs = 0 if op == OP_J2 else nq * 2 * nn * d
    return {"geometry": geometry, "coords": coords, "grad": grad, "prod": prod, "rhs": rhs}


def j2_point_flops(plastic, iters):
    """FP64 arithmetic of the J2 update at one point beyond the geometry (FMA = 2, exp / div / sqrt = 1).

    displacement gradient from the modal form of the nodal displacements: J_u
    (its columns shared by the points as J's: 108 FMA per element, 27 flop per
    point), grad u = J_u C^T (27 FMA), times 1/det J (1 div + 9 mul);
    strain, trace and deviator 9; trial stress 2 mu (e_dev - eps_p) 12, its
    norm 13, sigma_y(alpha_n) 5, the yield test 2; an elastic point's stress
    4.  A plastic point adds 20 per Newton iteration (alpha, sigma_y and its
    slope with one exp, g, g', the update with one div) and 47 for the flow
    direction, stress, plastic strain, alpha and the tangent factors.
    """
    base = 27 + 54 + 10 + 9 + 12 + 13 + 5 + 2
    return base + (47 + 20 * iters if plastic else 4)


def assembly_work(type_counts, n_nodes, nnz_node, op, precision, nq_of=None, k_varies=False, j2=None):
    """FP64 flops, FP32 flops and algorithmic bytes of one assembly.

    type_counts: {element type: count}; nnz_node: node-level nonzeros of the
    pattern (the scalar count is d^2 times it); precision 0 = FP64 (every
    flop on the FP64 pipe), 1 = FP32-integrate (geometry, coordinates, the
    J2 update and the accumulation in FP64, the rest in FP32), 2 =
    FP32-adaptive (as 1 with the geometry in FP32); nq_of: points
    of each type's rule (default: the degree-2 rules, tet 4, pyr 8, prism 6,
    hex 8); j2: dict(points, plastic_points, newton_iters) summed over the
    mesh for the J2 operator (hex8 only).

    Accumulation: an entry with c contributions takes c - 1 FP64 adds; A is
    symmetric, so the (a <= b) blocks of every element are counted, against
    the (nnz_node + n_nodes) / 2 node pairs (i <= j) of the pattern; b takes
    sum(nn) - n_nodes per component.
    Bytes: A written once (8 per scalar nonzero), b written once, coordinates
    (24 per node), scalar row starts (8 per row), connectivity (4 nn) and the
    node map (4 nn^2) per element read once; J2 also reads the displacements
    (24 per node) and reads and writes the state (8 points x 7 values x 8
    bytes each way per element).
    """
    nq_of = nq_of or {0: 4, 1: 8, 2: 6, 3: 8}
    d = 1 if op == OP_DIFFUSION else 3
    f64 = f32 = 0
    parts = {"geometry": 0, "accumulate": 0, "integrate": 0, "j2_update": 0}
    n_elems = sum(type_counts.values())
    sum_pairs = sum(c * NODES_PER_TYPE[t] * (NODES_PER_TYPE[t] + 1) // 2 for t, c in type_counts.items())
    sum_nn = sum(c * NODES_PER_TYPE[t] for t, c in type_counts.items())
    sum_nn2 = sum(c * NODES_PER_TYPE[t] ** 2 for t, c in type_counts.items())
    for t, c in type_counts.items():
        if not c:
            continue
        w = element_flops(t, op, nq_of[t], k_varies)
        parts["geometry"] += c * (w["geometry"] + w["coords"])
        if op == OP_J2:
            assert t == 3, "the J2 workload is hex8"
            parts["geometry"] += c * 72              # modal transform of the displacements
        parts["integrate"] += c * (w["grad"] + w["prod"] + w["rhs"])
    if op == OP_J2:
        j = j2 or {}
        plastic_extra = j2_point_flops(True, 0) - j2_point_flops(False, 0)
        parts["j2_update"] = (j.get("points", 0) * j2_point_flops(False, 0)
                              + j.get("plastic_points", 0) * plastic_extra + 20 * j.get("newton_iters", 0))
    parts["accumulate"] = d * d * (sum_pairs - (nnz_node + n_nodes) // 2) + d * (sum_nn - n_nodes)
    f64 = parts["geometry"] + parts["accumulate"] + parts["j2_update"]
    if precision == 0:
        f64 += parts["integrate"]
    else:
        f32 = parts["integrate"]
    if precision == 2:
        # FP32-adaptive: the geometry of undistorted elements is FP32 (the few
        # distorted ones redone in FP64 are not counted)
        f64 -= parts["geometry"]
        f32 += parts["geometry"]
    nnz = d * d * nnz_node
    by = 8 * nnz + n_nodes * (24 + 8 * d + 8 * d) + 4 * sum_nn + 4 * sum_nn2
    if op == OP_J2:
        by += 24 * n_nodes + n_elems * 2 * 8 * 7 * 8
    return {"fp64": f64, "fp32": f32, "bytes": by, "parts": parts, "elements": n_elems}


def fp64_peak_flops():
    """The FP64 rate the roofline uses: the measured FMA rate where a probe ran, else nominal."""
    return NOMINAL_FP64_TFLOPS * 1e12


def step_roofline(work, ms, peaks):
    """T_roof = max(FP64 flops / P64, FP32 flops / P32, bytes / HBM) against the measured step time."""
    t = {"fp64": work["fp64"] / peaks["fp64"], "fp32": work["fp32"] / peaks["fp32"],
         "hbm": work["bytes"] / peaks["hbm"]}
    bound = max(t, key=t.get)
    t_roof = t[bound]
    sec = ms * 1e-3
    ach = {"fp64": (work["fp64"] / sec / 1e9, "GFLOP/s (FP64)"), "fp32": (work["fp32"] / sec / 1e9, "GFLOP/s (FP32)"),
           "hbm": (work["bytes"] / sec / 1e9, "GB/s")}
    return {"bound": "hbm" if bound == "hbm" else "alu", "resource": bound, "achieved": ach[bound][0],
            "peak": peaks[bound] / 1e9, "unit": ach[bound][1], "frac": t_roof * 1e3 / ms, "t_roof_ms": t_roof * 1e3,
            "fp64_ms": t["fp64"] * 1e3, "fp32_ms": t["fp32"] * 1e3, "hbm_ms": t["hbm"] * 1e3, "ms": ms}


def record_bytes(n_elems):
    """FP32 geometry records: 208 values of 4 bytes per element."""
    return n_elems * 208 * 4


# ---------------------------------------------------------------------------
# multi-rank timing (one replica per rank, no data-path collective)
# ---------------------------------------------------------------------------

def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank gets it); identity on one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units all ranks processed per second of the slowest rank (weak scaling)."""
    return world * units_per_rank / (ms * 1e-3)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    """The engine's arm: every assembly variant, the product and the finite-strain operator
    on one replica per rank, the end-to-end pipeline, then the headline JSON line on
    rank 0."""
    import torch
    from paper_1805_03949_gb300 import fea

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    mesh = hex_cube_mesh(args.n)
    t0 = time.perf_counter()
    sysm = fea.System.from_mesh(mesh, 3, device=dev, with_cols=True)
    torch.cuda.synchronize()
    pattern_s = time.perf_counter() - t0
    nnz = sysm.A.numel()
    E, N = sysm.n_elems, sysm.n_nodes

    variants = variant_operators(fea)
    # results sampled for the error report: every dof row of ~30 seeded nodes,
    # copied to the host after each variant's timed region
    check = rank == 0 and not args.no_oracle
    rp_h = sysm.row_ptr.cpu().numpy() if check else None
    nodes = sample_hex_nodes(args.n, 11) if check else None
    snaps = {}
    if args.block_nodes:
        fea.fea_mesh_set_rows_block(sysm.handle, args.block_nodes)
    if args.block_elems:
        fea.fea_mesh_set_block_elems(sysm.handle, args.block_elems)
    if args.pipe_split:
        fea.fea_mesh_set_pipe_split(sysm.handle, args.pipe_split)
    if args.only:
        keep = set(args.only.split(",")) | {"fp64_atomic"}
        variants = {k: v for k, v in variants.items() if k in keep}
    plan_s = {}
    results = {}
    clocks = ClockSampler(local_rank, args.clocks_dir)
    clocks_started = False
    tuned = {}
    for name, op in variants.items():
        fea.set_events(op, None)
        t_first = time.perf_counter()
        sysm.assemble(op)                            # first call builds any plan the variant needs
        sysm.check()
        plan_s[name] = time.perf_counter() - t_first
        fixed = (name.endswith("rows") and args.block_nodes) or (name.endswith("block") and args.block_elems)
        if name in TUNED_VARIANTS and not args.no_tune and not fixed:
            # block sizes, the producer/consumer split, subdomain size: timed by the engine's autotuner
            t0 = time.perf_counter()
            tuned[name] = fea.fea_autotune(op, sysm.handle, sysm.row_ptr, sysm.node_map, sysm.A, sysm.b, 5)
            tuned[name]["seconds"] = time.perf_counter() - t0
        nk = fea.fea_assemble_launches(op, sysm.handle)     # every kernel of the step
        # block-task plans clear the rows of A they add to with one kernel,
        # inside the zeroing interval of the events below
        post = nk - 1 if name.endswith("block") else nk
        steps = args.steps if name.startswith("fp32") else max(3, min(args.steps, 5))
        # one set of profiling events per timed step: events[0] before zeroing, [1] after,
        # [2 + j] after the j-th kernel after the zeroing
        ev_steps = [[torch.cuda.Event(enable_timing=True) for _ in range(2 + post)] for _ in range(steps)]
        for evs in ev_steps:
            for e in evs:
                e.record()
        for _ in range(max(0, args.warmup - 1)):
            sysm.assemble(op)
        sysm.check()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        if not clocks_started:
            clocks.start()
            clocks_started = True
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record()
        for k in range(steps):
            fea.set_events(op, ev_steps[k])
            sysm.assemble(op)
        end.record()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        total_ms = start.elapsed_time(end)
        mean = lambda xs: sum(xs) / len(xs)
        kern_ms = mean([evs[1].elapsed_time(evs[-1]) for evs in ev_steps])
        zero_ms = mean([evs[0].elapsed_time(evs[1]) for evs in ev_steps])
        # dominant kernel: the last kernel of the step (tile / task kernel); a
        # colored step is one tile launch per color class, all counted
        if "color" in name:
            main_ms = kern_ms
        else:
            main_ms = mean([evs[-2].elapsed_time(evs[-1]) for evs in ev_steps])
        # geometry pass (ROWS / BLOCK): the kernels between the zeroing and the task kernel
        geo_ms = mean([evs[1].elapsed_time(evs[-2]) for evs in ev_steps]) if post > 1 and "color" not in name else 0.0
        fea.set_events(op, None)
        sysm.check()
        total_ms = max_over_ranks(total_ms, dist, dev)
        results[name] = dict(ms_per_step=total_ms / steps, kernel_ms=kern_ms, zero_ms=zero_ms, main_ms=main_ms,
                             geo_ms=geo_ms, launches=nk, post_launches=post, steps=steps)
        if check:
            snaps[name] = snapshot_rows(sysm, nodes, rp_h)
    clk = clocks.stop()
    # the assembled operator applied to a vector (partial-row product, Sec. 3.1),
    # on the system the last variant assembled
    spmv = None
    if rank == 0:
        x = torch.randn(sysm.b.numel(), dtype=torch.float64, device=dev)
        y = torch.empty_like(x)
        sp_ms = _time_calls(lambda: fea.fea_spmv(sysm.handle, 3, sysm.row_ptr, sysm.A, x, y), 20)
        sp_err = None
        if check:
            # the product's own rounding: sampled rows against the host FP64
            # product of the same A (normwise: over sum_j |a_ij x_j|)
            import torch as _t
            xh = x.cpu().numpy()
            rows = np.concatenate([3 * nodes + c for c in range(3)])
            worst = 0.0
            for r in rows:
                lo, hi = int(rp_h[r]), int(rp_h[r + 1])
                a = sysm.A[lo:hi].cpu().numpy()
                cols = sysm.col_idx[lo:hi].cpu().numpy()
                ax = a * xh[cols]
                worst = max(worst, abs(float(y[r].item()) - float(ax.sum())) / float(np.abs(ax).sum()))
            sp_err = {"y_normwise": worst, "rows": int(len(rows)),
                      "reference": "host FP64 product of the same A, sampled rows"}
        sp_bytes = algorithmic_bytes_spmv(N, nnz)
        hbm_pk, _ = _peaks()
        # one FP64 FMA per stored value: on GB300 the FP64 pipe bounds the product
        # about as tightly as HBM does, so both fractions are reported
        p64 = NOMINAL_FP64_TFLOPS * 1e12
        spmv = {"ms": sp_ms, "algorithmic_bytes": sp_bytes, "achieved_gbs": sp_bytes / (sp_ms * 1e-3) / 1e9,
                "peak_gbs": hbm_pk, "frac": sp_bytes / (sp_ms * 1e-3) / 1e9 / hbm_pk,
                "fp64_gflops": 2 * nnz / (sp_ms * 1e-3) / 1e9, "fp64_frac": 2 * nnz / (sp_ms * 1e-3) / p64,
                "floor_ms": {"hbm": sp_bytes / (hbm_pk * 1e9) * 1e3, "fp64": 2 * nnz / p64 * 1e3},
                "bytes": "A 8 nnz, node columns 4 nnz/9, node row starts, row_ptr (one per node), x and y once",
                "error": sp_err}
    # the finite-strain solid (Sec. 2.2, neo-Hookean reading) on the same mesh:
    # the Newton Jacobian and internal force at a smooth deformation
    neo = None
    if rank == 0:
        from paper_1805_03949_gb300 import meshgen as mg
        U = mg.fourier_displacement(mesh.coords, 0.004, seed=6) + 0.05 * mesh.coords[:, [1, 2, 0]]
        u_d = torch.tensor(U.reshape(-1), device=dev)
        neo = {"deformation": "fourier_displacement(0.004, seed 6) + 0.05 (y, z, x): strains of several %"}
        nh_nodes = sample_hex_nodes(args.n, 13, count=12)
        for name, prec, steps in (("fp32_atomic", 1, 10), ("fp64_atomic", 0, 3)):
            op = fea.make_operator(kind=fea.FEA_OP_NEOHOOKE, precision=prec, u=u_d, young=1.0, poisson=0.3)
            ms = _time_calls(lambda: sysm.assemble(op), steps)
            sysm.check()
            neo[name] = {"ms": ms, "elements_per_s": E / (ms * 1e-3)}
            if check:
                neo[name]["_snap"] = snapshot_rows(sysm, nh_nodes, rp_h)
        neo["_U"] = U
    fp32 = [k for k in results if k.startswith("fp32_")]
    head = args.variant if args.variant in results else min(fp32, key=lambda k: results[k]["ms_per_step"])

    # end to end through the C-ABI with host buffers: every step copies its
    # input (node coordinates, pinned) to the device, assembles, and reads its
    # result (A and b) back to pinned host memory.  Two steps are in flight:
    # the compute stream assembles step k into device buffer k % 2 while the
    # copy stream reads step k - 1 back (the read-back, 4.2 GB at the link's
    # ~190 GB/s, is the longest part); a buffer is reused only after its
    # read-back finished.
    op = variants[head]
    fea.set_events(op, None)
    host_numa, numa_rates = _bind_host_to_gpu_numa(dev.index if dev.index is not None else 0)
    coords_h = torch.from_numpy(mesh.coords.reshape(-1)).pin_memory()
    coords_d = torch.empty_like(coords_h, device=dev)
    A_d = [sysm.A, torch.empty_like(sysm.A)]
    b_d = [sysm.b, torch.empty_like(sysm.b)]
    A_h = torch.empty(nnz, dtype=torch.float64).pin_memory()
    b_h = torch.empty(sysm.b.numel(), dtype=torch.float64).pin_memory()
    comp, cp = torch.cuda.current_stream(), torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_step(k):
        j = k % 2
        if k >= 2:
            comp.wait_event(done[j])
        coords_d.copy_(coords_h, non_blocking=True)
        fea.fea_mesh_set_coords(sysm.handle, coords_d)
        fea.fea_assemble(op, sysm.handle, sysm.row_ptr, sysm.node_map, A_d[j], b_d[j])
        ready[j].record(comp)
        cp.wait_event(ready[j])
        with torch.cuda.stream(cp):
            A_h.copy_(A_d[j], non_blocking=True)
            b_h.copy_(b_d[j], non_blocking=True)
        done[j].record(cp)

    # five timed windows of e2e_steps steps each, the median reported: the
    # host link is shared, and its rate into pinned memory was seen to halve
    # for whole windows, which would otherwise set the figure
    e2e_steps = max(3, min(args.steps, 8))
    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    windows = []
    for _ in range(5):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(comp)
        for k in range(e2e_steps):
            e2e_step(k)
        comp.wait_stream(cp)
        s1.record(comp)
        torch.cuda.synchronize()
        windows.append(s0.elapsed_time(s1) / e2e_steps)
    e2e_ms = float(statistics.median(windows))
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    sysm.check()

    if rank == 0:
        r = results[head]
        pk = measured_peaks(fea)
        hbm, peak_kind = pk["hbm"] / 1e9, pk["hbm_source"]
        by = algorithmic_bytes(N, E, nnz)
        fl = algorithmic_flops_hex_elasticity(E, N, nnz)
        p64 = pk["fp64"]
        # whole step of every variant: T_roof = max(FP64 flops / P64, FP32 flops / P32, bytes / HBM)
        step_roofs = {k: step_roofline(assembly_work({3: E}, N, nnz // 9, OP_ELASTICITY, VARIANTS[k][0]),
                                       v["ms_per_step"], pk) for k, v in results.items()}
        step_roof = step_roofs[head]
        # dominant kernel of the step, against the roofline that bounds it
        kind = head.split("_", 1)[1]
        fused = kind == "block" and r["post_launches"] == 1   # the geometry runs inside the task kernel
        p64_note = {"peak_source": pk["fp64_source"], "peak_nominal": NOMINAL_FP64_TFLOPS * 1e3}
        if kind in ("rows", "block") and not fused and r["geo_ms"] > r["main_ms"]:
            k_name, k_ms = "k_geometry", r["geo_ms"]
            roof = dict({"bound": "alu", "achieved": fl["fp64_geometry"] / (k_ms * 1e-3) / 1e9, "peak": p64 / 1e9,
                         "unit": "GFLOP/s (FP64)", "work": "FP64 geometry"}, **p64_note)
        elif kind in ("rows", "block") and not fused:
            k_name, k_ms = DOMINANT_KERNEL[kind], r["main_ms"]
            plan = fea.fea_rows_plan_info(sysm.handle) if kind == "rows" else {"bytes": 0}
            kb = 8 * nnz + N * 3 * 16 + record_bytes(E) + plan.get("bytes", 0)
            roof = {"bound": "hbm", "achieved": kb / (k_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                    "peak_source": peak_kind, "algorithmic_bytes": kb}
        else:
            k_name, k_ms = DOMINANT_KERNEL.get(kind, head), r["main_ms"]
            # the FP64 adds of the accumulation run on the SMs, except under the
            # atomic scatter, whose adds the L2 atomic units perform
            on_sm = kind != "atomic"
            f64 = fl["fp64"] if on_sm else fl["fp64_geometry"]
            if "fp32_" in head and f64 / p64 > by / (hbm * 1e9):
                roof = dict({"bound": "alu", "achieved": f64 / (k_ms * 1e-3) / 1e9, "peak": p64 / 1e9,
                             "unit": "GFLOP/s (FP64)", "work": "FP64 geometry + the minimal FP64 accumulation adds"
                             if on_sm else "FP64 geometry"}, **p64_note)
            else:
                roof = {"bound": "hbm", "achieved": by / (k_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "peak_source": peak_kind, "algorithmic_bytes": by}
        kcfg = (k_name.split()[0],)
        if kind == "block":
            t = tuned.get(head, {})
            kcfg += (t.get("block_elems", args.block_elems or 64), t.get("producer_warps", args.pipe_split or 6))
        roof.update(frac=roof["achieved"] / roof["peak"], kernel=k_name, kernel_ms=k_ms,
                    traffic=TRAFFIC_BYTES.get(kcfg) if args.n == 128 else None,
                    kernel_config=list(kcfg[1:]) if len(kcfg) > 1 else None)
        if "peak_nominal" in roof:
            roof["frac_nominal"] = roof["achieved"] / roof["peak_nominal"]
        line = {
            "metric": METRIC,
            "value": whole_job_rate(E, world, r["ms_per_step"]),
            "unit": "elements/s",
            "n_gpus": world,
            "steps": r["steps"],
            "warmup": args.warmup,
            "ms_per_step": r["ms_per_step"],
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 integrate + f64 accumulate" if "fp32" in head else "f64",
            "data": "synthetic (seeded jittered hex8 cube; the paper's meshes are not available)",
            "config": {"workload": workload_name(args.n),
                       "variant": head, "l2": "inputs larger than L2 (A alone is 4.1 GB)",
                       "parallelism": f"replicas x{world} (partial-row, no exchange)"},
            "roofline": roof,
            "step_roofline": step_roof,
            "peaks": {k: v for k, v in pk.items()},
            "comparator": {"variant": "fp64_atomic",
                           "value": world * E / (results["fp64_atomic"]["ms_per_step"] * 1e-3),
                           "ms_per_step": results["fp64_atomic"]["ms_per_step"],
                           "kernel_ms": results["fp64_atomic"]["kernel_ms"]},
            "variants": {k: {"ms_per_step": v["ms_per_step"], "zero_ms": v["zero_ms"], "kernels_ms": v["kernel_ms"],
                             "main_kernel_ms": v["main_ms"], "geometry_ms": v["geo_ms"],
                             "launches_per_step": v["launches"],
                             "elements_per_s": E / (v["ms_per_step"] * 1e-3),
                             "step_roofline": step_roofs[k]} for k, v in results.items()},
            "pattern_build_s": pattern_s,
            "first_call_s": plan_s,
            "autotuned": tuned,
            "rows_plan": fea.fea_rows_plan_info(sysm.handle),
            "spmv": spmv,
            "neohooke": neo,
            "clocks": clk,
            "e2e": {"value": world * E / (e2e_ms * 1e-3), "unit": "elements/s",
                    "h2d_bytes_per_step": int(coords_h.numel() * 8),
                    "d2h_bytes_per_step": int((A_h.numel() + b_h.numel()) * 8),
                    "ms_per_step_windows": [round(w, 3) for w in windows],
                    "host_numa_node": host_numa,
                    "d2h_gbs_by_numa_node": {str(k): round(v, 1) for k, v in numa_rates.items()}},
            "gpu_launches": r["launches"] * r["steps"],
        }
        nh_snaps = {k: neo[k].pop("_snap") for k in list(neo) if isinstance(neo[k], dict) and "_snap" in neo[k]}
        nh_U = neo.pop("_U")
        if not (args.no_cpu_baseline or args.no_oracle):
            line["cpu_baseline"] = cpu_baseline(args)
        if check:
            # oracle leg: the error of every variant's sampled rows (after every timed region)
            ref = CpuBaselineLeg.rows(mesh, nodes, OP_ELASTICITY, young=1.0, poisson=0.3)
            errs = {k: row_errors(sn, ref, 1e-12 if VARIANTS[k][0] == 0 else 1e-5) for k, sn in snaps.items()}
            sample = f"every dof row of {len(nodes)} seeded nodes (corners, edges, faces, interior), oracle rows"
            line["error"] = dict(errs[head], sample=sample)
            line["errors"] = errs
            if nh_snaps:
                nh_ref = CpuBaselineLeg.nh_rows(mesh, nh_U, nh_nodes)
                for k, sn in nh_snaps.items():
                    neo[k]["error"] = row_errors(sn, nh_ref, 1e-12 if k.startswith("fp64") else 1e-5)
        if world == 1 and args.workloads:
            sysm.close()
            torch.cuda.empty_cache()
            line["workloads"] = other_workloads(args, dev, pk)
        print(json.dumps(line), flush=True)
    sysm.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the other workloads (one GPU, after the headline line's measurement)
# ---------------------------------------------------------------------------

def _node_cpus(node: int) -> set:
    cpus = set()
    for part in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
        if part:
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def _bind_host_to_gpu_numa(device_index: int):
    """Run this process on the CPUs of the NUMA node whose memory the GPU
    reads back fastest, so that the pinned host buffers allocated next (first
    touch) sit next to the GPU's link.  Every node with CPUs is tried: bound
    to its CPUs, a 256 MB pinned buffer is allocated and a device-to-host copy
    timed (the PCI function's numa_node in sysfs does not always name the
    socket that serves a Grace-attached GPU).  Returns (node, {node: GB/s}),
    or (None, {}) when sysfs lists no node (nothing changes)."""
    import torch
    try:
        nodes = sorted(int(d[4:]) for d in os.listdir("/sys/devices/system/node")
                       if d.startswith("node") and d[4:].isdigit())
        nodes = [n for n in nodes if _node_cpus(n)]
    except (OSError, ValueError):
        return None, {}
    if not nodes:
        return None, {}
    dev = torch.device("cuda", device_index)
    rates = {}
    src = torch.empty(32 << 20, dtype=torch.float64, device=dev)
    for node in nodes:
        try:
            os.sched_setaffinity(0, _node_cpus(node))
        except OSError:
            continue
        host = torch.empty(src.numel(), dtype=torch.float64).pin_memory()
        host.copy_(src)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            host.copy_(src, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        rates[node] = 3 * src.numel() * 8 / (a.elapsed_time(b) * 1e-3) / 1e9
        del host
    del src
    if not rates:
        return None, {}
    best = max(rates, key=rates.get)
    os.sched_setaffinity(0, _node_cpus(best))
    return best, rates


def _time_calls(fn, steps, warmup=2):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(statistics.median(ts))


def schedule_study(fea, s, base, counts, types, X, dev, steps, chunk, run=None, grid_fn=None, snap=None):
    """Persistent schedules of one workload: work stealing (whose per-item timings train the
    cost model), static LPT queues packed by the MLP's predictions or by Gauss-point weights, the
    same queues with stealing as the fallback once a CTA's own queue is empty, and stealing in
    predicted-cost order (largest first).  snap(name) is called after each schedule's timed calls
    (results sampled for the error report)."""
    import torch
    from paper_1805_03949_gb300 import meshgen as mg
    run = run or s.assemble
    grid_fn = grid_fn or fea.fea_persistent_grid
    snap = snap or (lambda name: None)
    item_ns = torch.zeros(len(counts), dtype=torch.int64, device=dev)
    steal = fea.make_operator(schedule=fea.FEA_SCHED_STEAL, chunk=chunk, item_ns=item_ns, **base)
    out = {"persistent_steal": _time_calls(lambda: run(steal), steps)}
    s.check()
    snap("persistent_steal")
    y = torch.log(item_ns.to(torch.float32) / torch.tensor(counts, device=dev, dtype=torch.float32))
    h = fea.fea_costmodel_create(6, mg.mlp_initial_params(6).astype(np.float32))
    t0 = time.perf_counter()
    fea.fea_costmodel_fit_scaler(h, X, y)
    loss = float(fea.fea_costmodel_train(h, X, y, 600, 1e-2).item())
    pred = fea.fea_costmodel_predict(h, X).cpu().numpy().astype(np.float64)
    train_s = time.perf_counter() - t0
    fea.fea_costmodel_destroy(h)
    grid = grid_fn(steal, s.handle)
    costs = {"mlp": np.exp(pred) * counts,
             "gauss_points": counts * np.array([4, 8, 6, 8])[types].astype(np.float64)}
    for name, cost in costs.items():
        q, off, _ = fea.fea_pack_lpt(cost, grid)
        qd, od = torch.tensor(q, device=dev), torch.tensor(off, device=dev)
        for mode, suffix in ((fea.FEA_SCHED_QUEUES, ""), (fea.FEA_SCHED_QUEUES_STEAL, "_steal")):
            op = fea.make_operator(schedule=mode, n_ctas=grid, queue=qd, queue_off=od, chunk=chunk, **base)
            out[f"{name}_queues{suffix}"] = _time_calls(lambda: run(op), steps)
            s.check()
            snap(f"{name}_queues{suffix}")
        # list scheduling in predicted-cost order: stealing takes the items
        # largest first (LPT order), so the tail holds the smallest ones
        order = torch.tensor(np.argsort(-cost, kind="stable").astype(np.int32), device=dev)
        op = fea.make_operator(schedule=fea.FEA_SCHED_STEAL, chunk=chunk, queue=order, **base)
        out[f"{name}_ordered_steal"] = _time_calls(lambda: run(op), steps)
        s.check()
        snap(f"{name}_ordered_steal")
    return out, {"train_loss": loss, "train_s": train_s, "epochs": 600, "items": len(counts), "chunk": chunk,
                 "grid": grid, "items_per_cta": len(counts) / grid,
                 "gain_static": out["gauss_points_queues"] / out["mlp_queues"] - 1.0,
                 "gain_with_steal": out["gauss_points_queues_steal"] / out["mlp_queues_steal"] - 1.0,
                 "gain_ordered_vs_gauss_points": out["gauss_points_ordered_steal"] / out["mlp_ordered_steal"] - 1.0,
                 "gain_ordered_vs_steal": out["persistent_steal"] / out["mlp_ordered_steal"] - 1.0}


def _type_counts(mesh):
    return {t: int(c) for t, c in enumerate(np.bincount(np.asarray(mesh.types), minlength=4)) if c}


def _rooflines(ms, work_of, pk):
    """Step roofline of every timed variant: work_of(variant) -> assembly_work(...)."""
    return {k: step_roofline(work_of(k), v, pk) for k, v in ms.items()}


def workload_poisson(dev, pk, check, steps=20):
    """Scalar Poisson P1 on 16^3 Kuhn tets (24,576 elements, 1-point rule, FP64): a
    correctness-sized problem that fits in L2, bounded by launch latency."""
    from paper_1805_03949_gb300 import fea, meshgen as mg
    mesh = mg.kuhn_tet_cube(16)
    s = fea.System.from_mesh(mesh, 1, device=dev, with_cols=False)
    try:
        kw = dict(kind=0, tet_rule=0, k0=1.0, k2=0.0, source=1.0)
        out, snaps = {}, {}
        for name, op in (("fp64_per_type", fea.make_operator(precision=0, **kw)),
                         ("fp32_per_type", fea.make_operator(precision=1, **kw)),
                         ("fp64_steal", fea.make_operator(precision=0, schedule=fea.FEA_SCHED_STEAL, **kw))):
            out[name] = _time_calls(lambda: s.assemble(op), steps)
            s.check()
            if check:
                snaps[name] = (s.A.cpu().numpy(), s.b.cpu().numpy())
        nnz_node = s.A.numel()
        prec = {"fp64_per_type": 0, "fp32_per_type": 1, "fp64_steal": 0}
        roof = _rooflines(out, lambda k: assembly_work(_type_counts(mesh), mesh.n_nodes, nnz_node, OP_DIFFUSION,
                                                       prec[k], nq_of={0: 1}), pk)
        res = {"workload": "Poisson P1, 16^3 Kuhn tets (24,576 elements, 4,913 nodes), 1-point rule, f = 1",
               "ms": out, "elements_per_s": {k: mesh.n_elems / (v * 1e-3) for k, v in out.items()},
               "roofline": roof, "bound_note": "the whole problem (about 2 MB) lives in L2: launch latency bounds it"}
        if check:
            res["error"] = CpuBaselineLeg.full_errors(mesh, snaps, prec, OP_DIFFUSION, tet_rule=0, k0=1.0, k2=0.0,
                                              source=1.0)
        return res
    finally:
        s.close()


def workload_hybrid(dev, pk, check, steps=5, n=100):
    """Hybrid tet/pyramid/prism/hex diffusion, k = 1 + x^2, degree-2 rules: per-type launches
    against one persistent launch over every type, scheduled by stealing or by packed queues."""
    from paper_1805_03949_gb300 import fea, meshgen as mg
    mesh = mg.hybrid_cube(n, 3)
    s = fea.System.from_mesh(mesh, 1, device=dev, with_cols=False)
    try:
        kw = dict(kind=0, tet_rule=1, k0=1.0, k2=1.0, source=1.0)
        nodes = sample_nodes(mesh.n_nodes, 3) if check else None
        rp_h = s.row_ptr.cpu().numpy() if check else None
        snaps = {}
        snap = (lambda name: snaps.__setitem__(name, snapshot_rows(s, nodes, rp_h))) if check else None
        out = {}
        for name, op in (("fp64_per_type", fea.make_operator(precision=0, **kw)),
                         ("fp32_per_type", fea.make_operator(precision=1, **kw))):
            out[name] = _time_calls(lambda: s.assemble(op), steps)
            s.check()
            if snap:
                snap(name)
        # the work-item size of the persistent launch: the autotuner's choice for stealing
        tune = fea.fea_autotune(fea.make_operator(precision=1, schedule=fea.FEA_SCHED_STEAL, chunk=128, **kw),
                                s.handle, s.row_ptr, s.node_map, s.A, s.b, 5)
        chunk = tune["chunk"]
        types, _, counts = fea.fea_work_items(s.handle, chunk)
        X = fea.fea_item_features(s.handle, chunk, len(counts), device=dev)
        sched, mlp = schedule_study(fea, s, dict(precision=1, **kw), counts, types, X, dev, steps, chunk,
                                    snap=(lambda n: snap("fp32_" + n)) if snap else None)
        mlp["autotuned"] = tune
        out.update({"fp32_" + k: v for k, v in sched.items()})
        nnz_node = s.A.numel()
        roof = _rooflines(out, lambda k: assembly_work(_type_counts(mesh), mesh.n_nodes, nnz_node, OP_DIFFUSION,
                                                       0 if k.startswith("fp64") else 1, k_varies=True), pk)
        res = {"workload": f"hybrid {n}^3 cube, {mesh.n_elems:,} elements (tet 40 / pyr 10 / prism 20 / hex 30 % "
                           "of the elements), diffusion k = 1 + x^2, degree-2 rules",
               "ms": out, "elements_per_s": {k: mesh.n_elems / (v * 1e-3) for k, v in out.items()}, "mlp": mlp,
               "roofline": roof}
        if check:
            ref = CpuBaselineLeg.rows(mesh, nodes, OP_DIFFUSION, tet_rule=1, k0=1.0, k2=1.0, source=1.0)
            res["error"] = {k: row_errors(sn, ref, 1e-12 if k.startswith("fp64") else 1e-5)
                            for k, sn in snaps.items()}
            res["error_sample"] = f"every row of {len(nodes)} seeded nodes, oracle rows"
        return res
    finally:
        s.close()


def workload_j2(dev, pk, check, steps=5, n=96):
    """Elastoplastic hex8 (J2 / Voce), 96^3, second load step from the committed first step: the
    plain per-type FP64 atomic assembly, FP32-integrate per type, and the persistent schedules."""
    import torch
    from paper_1805_03949_gb300 import fea, meshgen as mg
    amp = json.load(open(os.path.join(ROOT, "tests", "golden", "j2_amplitude.json")))["amplitude"]
    mesh, U = mg.j2_workload(n, amp)
    s = fea.System.from_mesh(mesh, 3, device=dev, with_cols=False)
    try:
        u = torch.tensor(U.reshape(-1), device=dev)
        st1 = torch.empty((mesh.n_elems, 8, 7), dtype=torch.float64, device=dev)
        yl = torch.empty((mesh.n_elems, 8), dtype=torch.uint8, device=dev)
        it = torch.empty((mesh.n_elems, 8), dtype=torch.uint8, device=dev)
        s.assemble(fea.make_operator(kind=fea.FEA_OP_J2, precision=0, u=0.5 * u, state_out=st1))
        st2 = torch.empty_like(st1)
        base = dict(kind=fea.FEA_OP_J2, u=u, state_in=st1, state_out=st2)
        nodes = sample_hex_nodes(n, 4, count=16) if check else None
        rp_h = s.row_ptr.cpu().numpy() if check else None
        snaps = {}
        snap = (lambda name: snaps.__setitem__(name, snapshot_rows(s, nodes, rp_h))) if check else None
        out = {}
        for name, op in (("fp64_per_type", fea.make_operator(precision=0, yield_out=yl, iters_out=it, **base)),
                         ("fp32_per_type", fea.make_operator(precision=1, **base))):
            out[name] = _time_calls(lambda: s.assemble(op), steps)
            s.check()
            if snap:
                snap(name)
        yield_frac = float(yl.float().mean().item())
        j2stats = {"points": 8 * mesh.n_elems, "plastic_points": int(yl.sum().item()),
                   "newton_iters": int(it.to(torch.int64).sum().item())}
        tune = fea.fea_autotune(fea.make_operator(precision=1, schedule=fea.FEA_SCHED_STEAL, chunk=32, **base),
                                s.handle, s.row_ptr, s.node_map, s.A, s.b, 5)
        chunk = tune["chunk"]
        types, _, counts = fea.fea_work_items(s.handle, chunk)
        X = fea.fea_item_features(s.handle, chunk, len(counts), u, st1, device=dev)
        sched, mlp = schedule_study(fea, s, dict(precision=1, **base), counts, types, X, dev, steps, chunk,
                                    snap=(lambda nm: snap("fp32_" + nm)) if snap else None)
        mlp["autotuned"] = tune
        out.update({"fp32_" + k: v for k, v in sched.items()})
        # the element-wise loop (no scatter): the Gauss-point update alone
        sig = torch.empty((mesh.n_elems, 8, 6), dtype=torch.float64, device=dev)
        loop = {"per_type": _time_calls(lambda: fea.fea_element_loop(fea.make_operator(**base), s.handle, sig), steps)}
        lsched, lmlp = schedule_study(fea, s, base, counts, types, X, dev, steps, chunk,
                                      run=lambda op: fea.fea_element_loop(op, s.handle, sig),
                                      grid_fn=fea.fea_element_loop_grid)
        loop.update(lsched)
        nnz_node = s.A.numel() // 9
        work = {p: assembly_work({3: mesh.n_elems}, mesh.n_nodes, nnz_node, OP_J2, p, j2=j2stats) for p in (0, 1)}
        roof = _rooflines(out, lambda k: work[0 if k.startswith("fp64") else 1], pk)
        # the element loop: the J2 update and its geometry and strain (FP64), state in and out
        loop_work = {"fp64": work[1]["parts"]["geometry"] + work[1]["parts"]["j2_update"], "fp32": 0,
                     "bytes": mesh.n_elems * (8 * 4 + 2 * 8 * 7 * 8 + 8 * 6 * 8) + mesh.n_nodes * (24 + 24)}
        loop_roof = {k: step_roofline(loop_work, v, pk) for k, v in loop.items()}
        res = {"workload": f"J2 / Voce hex8 {n}^3 jittered, {mesh.n_elems:,} elements, second load step "
                           f"(amplitude {amp:.4e}, {100 * yield_frac:.1f} % of Gauss points yield)",
               "ms": out, "elements_per_s": {k: mesh.n_elems / (v * 1e-3) for k, v in out.items()}, "mlp": mlp,
               "roofline": roof, "j2_work": j2stats,
               "element_loop": {"ms": loop, "elements_per_s": {k: mesh.n_elems / (v * 1e-3) for k, v in loop.items()},
                                "mlp": lmlp, "roofline": loop_roof}}
        if check:
            ref = CpuBaselineLeg.j2_rows(mesh, U, nodes)
            res["error"] = {k: row_errors(sn, ref, 1e-12 if k.startswith("fp64") else 1e-5)
                            for k, sn in snaps.items()}
            res["error_sample"] = f"every dof row of {len(nodes)} seeded nodes, oracle rows (both load steps)"
            elems = np.random.default_rng(8).choice(mesh.n_elems, size=256, replace=False)
            ei = torch.as_tensor(elems, device=dev)
            res["element_loop"]["error"] = dict(
                CpuBaselineLeg.j2_point_errors(mesh, U, elems, st2[ei].cpu().numpy(), sig[ei].cpu().numpy()),
                sample="256 seeded elements x 8 points, the oracle's own two steps")
        return res
    finally:
        s.close()


def workload_batch(dev, pk, check, steps=10):
    """256 tet4/hex8 elasticity meshes (log-uniform 1e3..2e5 elements), one graph-captured
    persistent launch, autotuned chunk and grid; aggregate rate and per-mesh latency."""
    from paper_1805_03949_gb300 import fea, meshgen as mg
    meshes = mg.batch_meshes(256, 5)
    systems = [fea.System.from_mesh(m, 3, device=dev, with_cols=False) for m in meshes]
    batch = None
    try:
        op = fea.make_operator(kind=1, precision=1, poisson=0.3)
        batch = fea.Batch(op, systems)
        tuned = batch.autotune(reps=2)
        batch.capture()
        ms = _time_calls(batch.assemble, steps)
        lat = batch.latency_ns().astype(np.float64) * 1e-6
        for s in systems:
            s.check()
        E = sum(m.n_elems for m in meshes)
        total = {"fp64": 0, "fp32": 0, "bytes": 0}
        for m, s in zip(meshes, systems):
            w = assembly_work(_type_counts(m), m.n_nodes, s.A.numel() // 9, OP_ELASTICITY, 1)
            for k in total:
                total[k] += w[k]
        res = {"workload": f"256 tet4/hex8 elasticity meshes, {E:,} elements, FP32-integrate, one CUDA graph "
                           "(zeroing kernel + persistent work-stealing launch)",
               "ms": ms, "elements_per_s": E / (ms * 1e-3), "autotuned": tuned,
               "roofline": step_roofline(total, ms, pk),
               "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                              "max": float(lat.max())}}
        if check:
            sizes = np.array([m.n_elems for m in meshes])
            pick = sorted({int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), int(np.argmax(sizes))})
            errs = {}
            for k in pick:
                nd = sample_nodes(meshes[k].n_nodes, 50 + k, count=8)
                sn = snapshot_rows(systems[k], nd)
                ref = CpuBaselineLeg.rows(meshes[k], nd, OP_ELASTICITY, tet_rule=1, young=1.0, poisson=0.3)
                errs[f"mesh{k}_{meshes[k].n_elems}"] = row_errors(sn, ref, 1e-5)
            res["error"] = errs
            res["error_sample"] = "the smallest, the median and the largest mesh: every row of 10 seeded nodes"
        return res
    finally:
        if batch is not None:
            batch.close()
        for s in systems:
            s.close()


def other_workloads(args, dev, pk):
    """Time the workloads named in --workloads (Poisson, mixed-element diffusion, J2, batch)."""
    out = {}
    wanted = [c for c in args.workloads.split(",") if c]
    check = not args.no_oracle
    for key, fn in (("poisson", workload_poisson), ("hybrid", workload_hybrid), ("j2", workload_j2),
                    ("batch", workload_batch)):
        if key in wanted:
            t0 = time.perf_counter()
            if key == "j2":
                out[key] = fn(dev, pk, check, n=args.j2_n)
            elif key == "hybrid":
                out[key] = fn(dev, pk, check, n=args.hybrid_n)
            else:
                out[key] = fn(dev, pk, check)
            out[key]["wall_s"] = time.perf_counter() - t0
            import torch
            torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# sampled results, copied to the host after a timed region (no oracle here)
# ---------------------------------------------------------------------------

def sample_hex_nodes(n, seed, count=24):
    """Corner, edge, face and centre nodes of an n^3 hex lattice, and `count` seeded ones."""
    m = n + 1
    idx = lambda i, j, k: i + m * (j + m * k)
    fixed = [idx(0, 0, 0), idx(n, n, n), idx(n, 0, 0), idx(0, n, min(5, n)), idx(min(3, n), 0, min(7, n)),
             idx(n, min(9, n), n // 2), idx(n // 2, n // 2, n // 2)]
    rnd = np.random.default_rng(seed).integers(0, m ** 3, size=count).tolist()
    return np.array(sorted(set(fixed + rnd)), dtype=np.int32)


def sample_nodes(n_nodes, seed, count=24):
    """The first and last node and `count` seeded ones."""
    rnd = np.random.default_rng(seed).integers(0, n_nodes, size=count)
    return np.unique(np.concatenate([rnd, [0, n_nodes - 1]])).astype(np.int32)


def snapshot_rows(system, nodes, rp_h=None):
    """Every dof row of the given nodes in the system's A, and their b entries, on the host."""
    import torch
    d = system.ndof
    if rp_h is None:
        rp_h = system.row_ptr.cpu().numpy()
    segs = [(int(rp_h[d * nd + c]), int(rp_h[d * nd + c + 1])) for nd in nodes for c in range(d)]
    idx = np.concatenate([np.arange(lo, hi) for lo, hi in segs]).astype(np.int64)
    vals = system.A[torch.as_tensor(idx, device=system.A.device)].cpu().numpy()
    bidx = np.array([d * nd + c for nd in nodes for c in range(d)], dtype=np.int64)
    bv = system.b[torch.as_tensor(bidx, device=system.b.device)].cpu().numpy()
    rows, o = [], 0
    for lo, hi in segs:
        rows.append(vals[o:o + hi - lo])
        o += hi - lo
    return {"nodes": np.asarray(nodes), "d": d, "rows": rows, "b": bv}


def row_errors(snap, ref_rows, bar):
    """Error of sampled rows against reference rows (the oracle's, one dict per node with
    vals / nvals [d, k d], b / sb [d]):
      normwise: max |a - r| / N, N the entry's normwise scale (entries with N = 0
                count |a| / max N); the metric the parity bars apply to;
      relative: max |a - r| / |r| over entries with |r| >= 1e-8 max over the row |r|;
    for A and b."""
    d = snap["d"]
    nw = rel = bnw = brel = 0.0
    n_ent = 0
    for k, r in enumerate(ref_rows):
        for c in range(d):
            a, v, nv = snap["rows"][k * d + c], r["vals"][c], r["nvals"][c]
            if len(a) != len(v):
                raise ValueError("sampled row and reference row differ in length")
            n_ent += len(v)
            diff = np.abs(a - v)
            pos = nv > 0
            if pos.any():
                nw = max(nw, float(np.max(diff[pos] / nv[pos])))
            if (~pos).any():
                nw = max(nw, float(np.max(np.abs(a[~pos]))) / max(float(nv.max()), 1e-300))
            big = np.abs(v) >= 1e-8 * np.abs(v).max()
            if big.any():
                rel = max(rel, float(np.max(diff[big] / np.abs(v[big]))))
            db = abs(float(snap["b"][k * d + c]) - r["b"][c])
            if r["sb"][c] > 0:
                bnw = max(bnw, db / r["sb"][c])
            if r["b"][c] != 0:
                brel = max(brel, db / abs(r["b"][c]))
    return {"A_normwise": nw, "A_relative": rel, "b_normwise": bnw, "b_relative": brel, "bar": bar,
            "within_bar": bool(nw <= bar and bnw <= bar), "rows": len(ref_rows) * d, "entries": n_ent}


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline, --impl reference, and the error of each result)
# ---------------------------------------------------------------------------

def _slab(mesh, layers, n):
    """The first `layers` cell layers (z) of the hex cube: a bounded sample of the workload."""
    from paper_1805_03949_gb300 import meshgen as mg
    E = layers * n * n
    nodes_used = (layers + 1) * (n + 1) ** 2
    return mg.Mesh(mesh.coords[:nodes_used].copy(), mesh.types[:E].copy(), mesh.conn_offsets[:E + 1].copy(),
                   mesh.conn[:8 * E].copy(), {"kind": "slab", "layers": layers})


def cpu_baseline(args, mesh=None, layers=None):
    """The FP64 oracle, as it stands, on the first `layers` cell layers of the workload (one thread)."""
    from oracle import oracle as O
    n = args.n
    mesh = mesh if mesh is not None else hex_cube_mesh(n)
    layers = layers or args.cpu_layers
    sub = _slab(mesh, layers, n)
    pat = O.pattern(sub, 3)
    t0 = time.perf_counter()
    O.assemble(sub, O.OP_ELASTICITY, pat=pat, young=1.0, poisson=0.3)
    dt = time.perf_counter() - t0
    return {"value": sub.n_elems / dt, "unit": "elements/s", "cores": 1, "kind": "oracle",
            "sample": f"first {layers} of {n} cell layers of the workload ({sub.n_elems} elements), "
                      f"single-thread FP64 oracle, element-index order, pattern excluded",
            "seconds": dt}


class CpuBaselineLeg:
    """The CPU-baseline leg: everything bench.py does with the oracle, on the host,
    after every timed GPU region -- timing the oracle on a bounded sample of the
    workload (cpu_baseline) and recomputing sampled results, from which the error
    of each GPU result is reported.  Nothing else in the bench touches the oracle."""

    @staticmethod
    def full_errors(mesh, snaps, prec, op, **kw):
        """Oracle leg: the whole assembled system of a small workload against the oracle's."""
        from oracle import oracle as O
        ref = O.assemble(mesh, op, **kw)
        out = {}
        for k, (A, b) in snaps.items():
            pos = ref["NA"] > 0
            dA = np.abs(A - ref["A"])
            big = np.abs(ref["A"]) >= 1e-8 * np.abs(ref["A"]).max()
            bar = 1e-12 if prec[k] == 0 else 1e-5
            nw = max(float(np.max(dA[pos] / ref["NA"][pos])),
                     float(np.max(np.abs(A[~pos]), initial=0.0)) / float(ref["NA"].max()))
            bnw = float(np.max(np.abs(b - ref["b"]) / ref["Nb"]))
            out[k] = {"A_normwise": nw, "A_relative": float(np.max(dA[big] / np.abs(ref["A"][big]))),
                      "b_normwise": bnw, "b_relative": float(np.max(np.abs(b - ref["b"]) / np.abs(ref["b"]))),
                      "bar": bar, "within_bar": bool(nw <= bar and bnw <= bar), "entries": int(A.size),
                      "sample": "the whole system"}
        return out

    @staticmethod
    def rows(mesh, nodes, op, **kw):
        """Oracle leg: every dof row of the nodes, summed over all elements in index order."""
        from oracle import oracle as O
        return O.assemble_rows(mesh, nodes, op, **kw)

    @staticmethod
    def rows_from_elements(mesh, nodes, element_fn):
        """Oracle leg: rows of the nodes of a hex8 mesh (3 dofs per node) summed from
        per-element matrices; element_fn(e) -> dict(A, b, NA, Nb) of element e."""
        conn = np.asarray(mesh.conn).reshape(-1, 8)
        out = []
        for node in nodes:
            blocks = {}
            b = np.zeros(3)
            sb = np.zeros(3)
            for e, a in zip(*np.nonzero(conn == node)):
                r = element_fn(int(e))
                for bb in range(8):
                    j = int(conn[e, bb])
                    v, nv = blocks.get(j, (np.zeros((3, 3)), np.zeros((3, 3))))
                    blocks[j] = (v + r["A"][3 * a:3 * a + 3, 3 * bb:3 * bb + 3],
                                 nv + r["NA"][3 * a:3 * a + 3, 3 * bb:3 * bb + 3])
                b += r["b"][3 * a:3 * a + 3]
                sb += r["Nb"][3 * a:3 * a + 3]
            cols = sorted(blocks)
            vals = np.concatenate([blocks[j][0] for j in cols], axis=1)
            nvals = np.concatenate([blocks[j][1] for j in cols], axis=1)
            out.append({"cols": np.array(cols), "vals": vals, "nvals": nvals, "b": b, "sb": sb})
        return out

    @staticmethod
    def j2_rows(mesh, U, nodes):
        """Oracle leg: rows of the J2 tangent and internal force at displacement U after
        the committed step at 0.5 U (both steps taken by the oracle, per element)."""
        from oracle import oracle as O
        conn = np.asarray(mesh.conn).reshape(-1, 8)

        def elem(e):
            X, Ue = mesh.coords[conn[e]], U[conn[e]]
            st1 = O.j2_element(3, X, 0.5 * Ue)["state"]
            return O.j2_element(3, X, Ue, st1)
        return CpuBaselineLeg.rows_from_elements(mesh, nodes, elem)

    @staticmethod
    def nh_rows(mesh, U, nodes):
        """Oracle leg: rows of the finite-strain Jacobian and internal force at U."""
        from oracle import oracle as O
        conn = np.asarray(mesh.conn).reshape(-1, 8)
        return CpuBaselineLeg.rows_from_elements(mesh, nodes, lambda e: O.nh_element(3, mesh.coords[conn[e]], U[conn[e]],
                                                                       young=1.0, poisson=0.3))

    @staticmethod
    def j2_point_errors(mesh, U, elems, state, stress, young=1.0, poisson=0.3):
        """Oracle leg: the J2 update (state and stress of step 2 from the oracle's own
        step 1) on sampled hex elements, against the GPU's; per-point normwise errors
        with the scale S = max|eps_p| + |alpha| + max|sigma| / (2 mu) of the point."""
        from oracle import oracle as O
        from paper_1805_03949_gb300 import meshgen as mg
        conn = np.asarray(mesh.conn).reshape(-1, 8)[elems]
        sub = mg.Mesh(mesh.coords, np.full(len(elems), 3, dtype=np.uint8),
                      np.arange(len(elems) + 1, dtype=np.int64) * 8, conn.reshape(-1).astype(np.int32), {})
        r1 = O.j2_points(sub, 0.5 * U)
        r2 = O.j2_points(sub, U, r1["state"])
        mu = young / (2.0 * (1.0 + poisson))
        kappa = young / (3.0 * (1.0 - 2.0 * poisson))
        S = (np.abs(r2["state"][..., :6]).max(-1) + np.abs(r2["state"][..., 6])
             + np.abs(r2["stress"]).max(-1) / (2.0 * mu)).reshape(-1)
        ds = np.abs(state - r2["state"]).max(-1).reshape(-1)
        dsig = np.abs(stress - r2["stress"]).max(-1).reshape(-1)
        pos = S > 0
        return {"state_normwise": float(np.max(ds[pos] / S[pos])),
                "stress_normwise": float(np.max(dsig[pos] / ((3 * kappa + 2 * mu) * S[pos]))),
                "points": int(pos.size), "bar": 1e-12,
                "within_bar": bool(np.max(ds[pos] / S[pos]) <= 1e-12
                                   and np.max(dsig[pos] / ((3 * kappa + 2 * mu) * S[pos])) <= 1e-12)}


def workload_name(n: int) -> str:
    """The bench workload, named by what it is (both arms use this name).  The
    scalar system of an n^3 hex lattice with 3 dofs per node has
    9 (3 n + 1)^3 nonzeros: per axis a node couples with itself and its two
    lattice neighbours, 3 (n + 1) - 2 pairs."""
    return (f"hex8 linear elasticity, {n}^3 jittered cube (+-0.2h, PCG64 seed 2), "
            f"{n ** 3:,} elements, {9 * (3 * n + 1) ** 3:,} nonzeros, 2x2x2 Gauss")


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle timed on slabs of the workload (rank 0 only)."""
    if rank != 0:
        return
    mesh = hex_cube_mesh(args.n)
    vals, secs = [], []
    for _ in range(args.warmup):
        cpu_baseline(args, mesh, layers=1)
    for _ in range(args.steps):
        cb = cpu_baseline(args, mesh, layers=args.ref_layers)
        vals.append(cb["value"])
        secs.append(cb["seconds"])
    E = args.ref_layers * args.n * args.n
    ms = 1e3 * statistics.median(secs)
    v = statistics.median(vals)
    line = {"metric": METRIC, "value": v, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(args.n),
                       "sample": f"{args.ref_layers} cell layers ({E} elements) per step"},
            "cpu_baseline": {"value": v, "unit": "elements/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.ref_layers} of {args.n} cell layers per step"},
            "e2e": {"value": v, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_parser() -> argparse.ArgumentParser:
    """Command-line options of both arms."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="", help="headline variant (default: the fastest fp32 one)")
    ap.add_argument("--only", default="", help="comma list of variants to time (fp64_atomic always)")
    ap.add_argument("--block-nodes", type=int, default=0)
    ap.add_argument("--block-elems", type=int, default=0,
                    help="elements per block of the block-task scatter (no autotuning of the block-task variant)")
    ap.add_argument("--pipe-split", type=int, default=0, help="producer warps of the pipelined block-task kernel")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--cpu-layers", type=int, default=8)
    ap.add_argument("--ref-layers", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="time the default launch parameters")
    ap.add_argument("--j2-n", type=int, default=96, help="cells per edge of the elastoplastic workload (96)")
    ap.add_argument("--hybrid-n", type=int, default=100, help="cells per edge of the mixed-element workload (100)")
    ap.add_argument("--no-oracle", action="store_true",
                    help="skip every oracle step: the CPU baseline and the error of each result")
    ap.add_argument("--clocks-dir", default=tempfile.gettempdir(),
                    help="where the raw nvidia-smi clock samples of the timed region are written")
    ap.add_argument("--workloads", "--configs", dest="workloads", default="poisson,hybrid,j2,batch",
                    help="other workloads timed after the headline one (comma list of poisson, hybrid, j2, "
                         "batch; '' for none)")
    return ap


def main():
    """Run the arm --impl selects and print its JSON line."""
    ap = make_parser()
    args = ap.parse_args()
    unknown = sorted({v for v in args.only.split(",") if v} - set(VARIANTS))
    if unknown:
        ap.error(f"unknown --only variant(s) {', '.join(unknown)}; known: {', '.join(VARIANTS)}")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
