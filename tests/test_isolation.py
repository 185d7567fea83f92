"""The oracle is test infrastructure: the product path neither imports nor falls
back to it, and bench.py reaches it only from its CPU legs (no GPU needed)."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2511_06824_gb300")


def _imports(path):
    tree = ast.parse(open(path).read())
    out = set()
    for n in ast.walk(tree):
        if isinstance(n, ast.Import):
            out.update(a.name.split(".")[0] for a in n.names)
        elif isinstance(n, ast.ImportFrom) and n.module and n.level == 0:
            out.add(n.module.split(".")[0])
    return out


def test_package_does_not_import_the_oracle():
    for f in sorted(os.listdir(PKG)):
        if f.endswith(".py"):
            assert "oracle" not in _imports(os.path.join(PKG, f)), f


def test_cuda_sources_do_not_reference_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            text = open(os.path.join(csrc, f)).read()
            for line in text.splitlines():
                code = line.split("//")[0]
                assert "oracle" not in code, (f, line)
    assert "oracle" not in open(os.path.join(ROOT, "include", "gmaf.h")).read()


def test_oracle_shares_no_code_with_the_package():
    imps = _imports(os.path.join(ROOT, "oracle", "__init__.py"))
    assert "paper_2511_06824_gb300" not in imps
    c = open(os.path.join(ROOT, "oracle", "gmaf_oracle.c")).read()
    assert "#include \"gmaf" not in c and "csrc" not in c


def test_bench_reaches_the_oracle_only_from_its_cpu_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = {"oracle_sample", "run_reference", "cpu_baseline"}
    hits = []

    class V(ast.NodeVisitor):
        def __init__(self):
            self.stack = []

        def visit_FunctionDef(self, n):
            self.stack.append(n.name)
            self.generic_visit(n)
            self.stack.pop()

        def visit_Name(self, n):
            if n.id == "oracle":
                hits.append(tuple(self.stack))

        def visit_alias(self, n):
            if n.name.split(".")[0] == "oracle":
                hits.append(tuple(self.stack))

    V().visit(tree)
    assert hits
    for stack in hits:
        assert stack and stack[0] in allowed, stack


def test_missing_library_raises_instead_of_falling_back():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2511_06824_gb300 import gmaf\n"
            "try:\n"
            "    gmaf.load('/nonexistent/libgmaf.so')\n"
            "except OSError:\n"
            "    print('raised')\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.stdout.strip() == "raised", r.stdout + r.stderr
