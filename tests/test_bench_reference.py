"""The reference arm of bench.py (the oracle timed on the host cores) runs on
CPU and prints one JSON line carrying the same metric and workload name as
the GPU arm, for one process and for two ranks (only rank 0 prints); and the
bench's algorithmic counts against brute-force counts on small meshes."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, n=8):
    env = dict(os.environ, **(extra_env or {}))
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--n", str(n), "--ref-layers", "1"],
                         capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_prints_one_line_with_the_workload_name():
    import bench
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "elements/s" and d["higher_is_better"] is True
    assert d["metric"] == bench.METRIC
    assert d["config"]["workload"] == bench.workload_name(8)
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert (d["n_gpus"], d["steps"], d["warmup"], d["scaling"], d["vs_baseline"]) == (1, 1, 0, "weak", None)
    assert set(d["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert d["cpu_baseline"]["cores"] == 1 and d["cpu_baseline"]["unit"] == d["unit"]
    assert set(d["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert d["e2e"]["unit"] == d["unit"] and d["e2e"]["d2h_bytes_per_step"] == 0


def test_workload_name_counts_the_lattice_nonzeros():
    """9 (3n + 1)^3 is the nonzero count of the oracle's own pattern."""
    import bench
    from oracle import oracle
    from paper_1805_03949_gb300 import meshgen as mg
    for n in (1, 2, 5):
        rp, cols, _ = oracle.pattern(mg.hex_cube(n, 0.2, 2), 3)
        assert f"{len(cols):,} nonzeros" in bench.workload_name(n)


def test_other_ranks_print_nothing():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_fp64_accumulation_count_matches_brute_force():
    """The roofline's FP64 accumulation adds: for every entry of the upper 3x3
    blocks (i <= j) and of b, (contributions - 1), counted element by element
    on small meshes against the closed form in the bench."""
    import bench
    from paper_1805_03949_gb300 import meshgen as mg
    for n, jit in ((1, 0.0), (3, 0.2), (4, 0.1)):
        mesh = mg.hex_cube(n, jit, 2)
        conn = mesh.conn.reshape(-1, 8)
        contrib = {}
        bcount = np.zeros(mesh.n_nodes, dtype=np.int64)
        for e in conn:
            for a in range(8):
                bcount[e[a]] += 1
                for b in range(8):
                    i, j = int(e[a]), int(e[b])
                    if i <= j:
                        contrib[(i, j)] = contrib.get((i, j), 0) + 1
        # every element adds into 36 upper blocks (8 diagonal, 28 pairs), each
        # of 9 entries; an entry with c contributions takes c - 1 adds
        adds_A = 9 * sum(c - 1 for c in contrib.values())
        adds_b = 3 * int((bcount - 1).clip(min=0).sum())
        nnz = 9 * (3 * n + 1) ** 3
        fl = bench.algorithmic_flops_hex_elasticity(mesh.n_elems, mesh.n_nodes, nnz)
        assert fl["fp64_accumulate"] == adds_A + adds_b, n


def test_algorithmic_bytes_are_the_arrays_one_assembly_moves():
    """A written once, b written once, and the inputs read once: coordinates,
    scalar row starts, connectivity and the element-to-nonzero map, each
    counted from the arrays of a small hex mesh and the oracle's pattern."""
    import bench
    from oracle import oracle
    from paper_1805_03949_gb300 import meshgen as mg
    for n in (1, 3):
        mesh = mg.hex_cube(n, 0.2, 2)
        rp, cols, nmap = oracle.pattern(mesh, 3)
        b = np.zeros(3 * mesh.n_nodes)
        moved = (8 * len(cols) + b.nbytes + mesh.coords.astype(np.float64).nbytes + 8 * (len(rp) - 1)
                 + mesh.conn.astype(np.int32).nbytes + nmap.astype(np.int32).nbytes)
        assert bench.algorithmic_bytes(mesh.n_nodes, mesh.n_elems, len(cols)) == moved, n


def test_spmv_algorithmic_bytes_are_the_arrays_the_product_moves():
    """A, the node-level columns, the node and scalar row starts, x and y."""
    import bench
    from oracle import oracle
    from paper_1805_03949_gb300 import meshgen as mg
    for n in (1, 3):
        mesh = mg.hex_cube(n, 0.2, 2)
        rp_node, cols_node, _ = oracle.pattern(mesh, 1)
        rp, cols, _ = oracle.pattern(mesh, 3)
        x = np.zeros(3 * mesh.n_nodes)
        moved = (8 * len(cols) + cols_node.astype(np.int32).nbytes + rp_node.astype(np.int64).nbytes
                 + rp.astype(np.int64).nbytes + 2 * x.nbytes)
        assert bench.algorithmic_bytes_spmv(mesh.n_nodes, len(cols)) == moved, n
