"""The oracle and the CUDA path share no code: no module of one imports the other, the
seeded-input module imports neither, and no native source or header reads the oracle.  Only
tests, the smoke check and bench.py's CPU legs import the oracle."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1612_04488_gb300"


def _imports(path):
    tree = ast.parse(open(path).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def _py(folder):
    d = os.path.join(ROOT, folder)
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


def test_oracle_imports_nothing_of_the_package():
    for f in _py("oracle"):
        assert PKG not in _imports(f), f


def test_package_imports_nothing_of_the_oracle():
    for f in _py(PKG):
        assert "oracle" not in _imports(f), f
    src = os.path.join(ROOT, PKG, "csrc")
    for f in sorted(os.listdir(src)):
        for line in open(os.path.join(src, f), errors="replace"):
            if line.lstrip().startswith("#include"):
                assert "oracle" not in line, (f, line)


def test_seeded_inputs_import_neither_side():
    assert _imports(os.path.join(ROOT, PKG, "workloads.py")) <= {"numpy"}


def test_only_tests_smoke_and_bench_import_the_oracle():
    allowed = {os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")}
    for dirpath, dirnames, files in os.walk(ROOT):
        dirnames[:] = [d for d in dirnames if d not in (".git", "_work", "gpurun_out", "baseline", "tests",
                                                        "oracle", "__pycache__", "_build")]
        for f in files:
            p = os.path.join(dirpath, f)
            if f.endswith(".py") and p not in allowed:
                assert "oracle" not in _imports(p), p
