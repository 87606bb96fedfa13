"""The oracle is test infrastructure: the product package never imports or
loads it, and bench.py uses it only in its CPU-baseline and reference legs."""
import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports_oracle(node):
    for n in ast.walk(node):
        if isinstance(n, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in n.names):
            return True
        if isinstance(n, ast.ImportFrom) and (n.module or "").split(".")[0] == "oracle":
            return True
    return False


def test_product_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(ROOT, "paper_1201_6062_gb300", "**", "*.py"), recursive=True):
        tree = ast.parse(open(path).read())
        assert not _imports_oracle(tree), path
    for path in glob.glob(os.path.join(ROOT, "paper_1201_6062_gb300", "csrc", "*")):
        txt = open(path, errors="replace").read()
        assert "liboracle" not in txt and "orc_" not in txt, path


def test_bench_uses_the_oracle_only_in_its_cpu_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    users = {f.name for f in tree.body if isinstance(f, ast.FunctionDef) and _imports_oracle(f)}
    assert users <= {"cpu_baseline", "run_reference"}, users
    top = [n for n in tree.body if not isinstance(n, ast.FunctionDef)]
    assert not any(_imports_oracle(n) for n in top)
