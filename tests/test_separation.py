"""The oracle and the engine share no code (no GPU).

The engine package never imports the oracle, and the bench imports it only in
its CPU-baseline leg (the oracle's timing on the host and its recomputation of
sampled results for the error report).  The oracle takes nothing from the package but the
seeded input module (meshgen), and its C sources include only standard
headers.
"""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    """(module, enclosing top-level function or None) of every import in a file."""
    tree = ast.parse(open(path).read())
    out = []
    for top in tree.body:
        owner = top.name if isinstance(top, (ast.FunctionDef, ast.ClassDef)) else None
        for n in ast.walk(top):
            if isinstance(n, ast.Import):
                out += [(a.name, owner) for a in n.names]
            elif isinstance(n, ast.ImportFrom):
                mod = ("." * n.level) + (n.module or "")
                out += [(mod + a.name if n.module is None else mod, owner) for a in n.names]
    return out


def test_engine_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1805_03949_gb300")
    for f in glob.glob(os.path.join(pkg, "*.py")):
        for mod, _ in _imports(f):
            assert not mod.split(".")[0] == "oracle", (f, mod)
    for f in glob.glob(os.path.join(pkg, "csrc", "*")):
        assert "oracle" not in open(f).read().lower(), f


def test_bench_imports_the_oracle_only_for_the_cpu_baseline():
    """Only the CPU-baseline leg (the oracle timed on the host, and the oracle's
    recomputation of sampled results for the error report, both after every
    timed GPU region) imports the oracle."""
    owners = set()
    for mod, owner in _imports(os.path.join(ROOT, "bench.py")):
        if mod.split(".")[0] == "oracle":
            assert owner in ("cpu_baseline", "CpuBaselineLeg"), (mod, owner)
            owners.add(owner)
    assert owners == {"cpu_baseline", "CpuBaselineLeg"}


def test_oracle_takes_only_the_input_module_from_the_package():
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        for mod, _ in _imports(f):
            if mod.startswith("paper_1805_03949_gb300"):
                assert mod == "paper_1805_03949_gb300" or mod.endswith("meshgen"), (f, mod)
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.c")):
        for inc in re.findall(r"#include\s*([<\"][^>\"]+[>\"])", open(f).read()):
            assert inc.startswith("<"), (f, inc)
