"""The oracle and the CUDA path share no code: the oracle imports nothing of the
package but its seeded input generators, the package never imports the oracle,
the CUDA sources never include it, and outside tests/ the oracle is reached
only by the smoke check and the benchmark's CPU-baseline / reference leg."""

import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_0711_0999_gb300"


def imports(path):
    """(module, enclosing function name or None) for every import in a file."""
    tree = ast.parse(open(path).read(), path)
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)) else fn
            if isinstance(child, ast.Import):
                out.extend((a.name, fn) for a in child.names)
            elif isinstance(child, ast.ImportFrom) and child.module:
                out.append((child.module, fn))
                out.extend((f"{child.module}.{a.name}", fn) for a in child.names)
            visit(child, name)

    visit(tree, None)
    return out


def test_oracle_imports_only_the_input_generators_of_the_package():
    files = glob.glob(os.path.join(ROOT, "oracle", "*.py"))
    assert files
    for f in files:
        for mod, _ in imports(f):
            if mod.startswith(PKG):
                assert mod in (f"{PKG}.synth", f"{PKG}.synth.workload_sigma"), (f, mod)


def test_synth_holds_no_method_arithmetic_imports():
    for mod, _ in imports(os.path.join(ROOT, PKG, "synth.py")):
        assert not mod.startswith("oracle") and not mod.startswith(f"{PKG}."), mod


def test_package_never_imports_the_oracle():
    for f in glob.glob(os.path.join(ROOT, PKG, "*.py")):
        for mod, _ in imports(f):
            assert not mod.startswith("oracle"), (f, mod)
    for f in glob.glob(os.path.join(ROOT, PKG, "csrc", "*")):
        text = open(f, errors="replace").read()
        assert "oracle" not in text.lower(), f


def test_oracle_reached_only_by_smoke_and_the_cpu_legs_of_the_benchmark():
    allowed = {
        "__graft_entry__.py": {"smoke"},
        "bench.py": {"_oracle_points", "__init__"},  # OracleTimer.__init__: the host-core timing pool
    }
    for name, fns in allowed.items():
        for mod, fn in imports(os.path.join(ROOT, name)):
            if mod.startswith("oracle"):
                assert fn in fns, (name, mod, fn)


def test_nothing_outside_the_scratch_folder_names_it():
    # scratch work lives in a git-ignored folder; no source, test or script reads, imports or runs it
    skip = {".git", "_work", "gpurun_out", "baseline", "__pycache__", "_build"}
    hits = []
    for base, dirs, files in os.walk(ROOT):
        dirs[:] = [d for d in dirs if d not in skip]
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp", ".sh", ".txt", ".cfg", ".toml", ".ini")):
                path = os.path.join(base, f)
                if re.search(r"(?<![A-Za-z0-9_])_work(?![A-Za-z0-9_])", open(path, errors="replace").read()):
                    hits.append(os.path.relpath(path, ROOT))
    assert hits == [os.path.join("tests", "test_independence_cpu.py")], hits
