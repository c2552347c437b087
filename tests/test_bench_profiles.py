"""The bench's variant table, and the commands the ncu summaries record (no GPU).

Every summary under profiles/ names the command that produced it.  These
tests check that each recorded ncu command leaves the GPU clocks alone
(--clock-control none), and that it runs committed files only.  A bench
command must also still parse with the bench's own options, and every
variant it selects must exist.
"""
import os
import re
import shlex

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.endswith((".md", ".txt")))


def _commands(path):
    """Shell lines of the fenced blocks of a summary, continuations joined."""
    text = open(path).read()
    out = []
    for block in re.findall(r"```[^\n]*\n(.*?)```", text, re.S):
        for line in block.replace("\\\n", " ").splitlines():
            line = line.strip()
            if line.startswith(("ncu ", "python ")):
                out.append(line)
    return out


def test_every_summary_records_an_ncu_command():
    assert PROFILES
    for f in PROFILES:
        cmds = _commands(os.path.join(ROOT, "profiles", f))
        assert any(c.startswith("ncu ") for c in cmds), f


@pytest.mark.parametrize("name", PROFILES)
def test_recorded_commands_keep_clocks_and_run_committed_files(name):
    for cmd in _commands(os.path.join(ROOT, "profiles", name)):
        toks = shlex.split(cmd)
        if toks[0] == "ncu":
            i = toks.index("--clock-control")
            assert toks[i + 1] == "none", cmd
        assert "_work" not in cmd and "/root/" not in cmd, cmd
        if "python" not in toks:
            continue
        prog = toks[toks.index("python") + 1:]
        if prog[0] == "-c":
            assert "__graft_entry__" in prog[1], cmd
            continue
        if prog[0] == "-m":
            assert prog[1] == "pytest", cmd
            files = [t for t in prog[2:] if t.endswith(".py")]
            assert files and all(os.path.isfile(os.path.join(ROOT, t)) for t in files), cmd
            continue
        script = prog[0]
        assert os.path.isfile(os.path.join(ROOT, script)), cmd
        if script == "bench.py":
            args = bench.make_parser().parse_args(prog[1:])
            assert {v for v in args.only.split(",") if v} <= set(bench.VARIANTS), cmd
            assert set(filter(None, args.workloads.split(","))) <= {"hybrid", "j2", "batch"}, cmd


def test_variant_operators_match_the_table():
    from paper_1805_03949_gb300 import fea
    ops = bench.variant_operators(fea)
    assert list(ops) == list(bench.VARIANTS)
    scatter = {"ATOMIC": 0, "COLOR": 1, "BLOCK": 2, "ROWS": 3, "MULTIDEP": 4}
    for name, (prec, sc) in bench.VARIANTS.items():
        op = ops[name]
        assert (op.kind, op.precision, op.scatter) == (1, prec, scatter[sc]), name
        assert (op.young, op.poisson, op.chunk, op.schedule) == (1.0, 0.3, 0, 0), name
        assert name.startswith({0: "fp64_", 1: "fp32_", 2: "fp32a_"}[prec]), name
