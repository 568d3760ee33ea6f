"""The oracle and the CUDA path share no code (CPU only).

Neither side imports the other, the product package never reaches the
oracle, and the input generators (shared by both) import neither.  Checked on
the sources' import statements, so a later edit that crosses the line fails
here."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read())
    out = set()
    for n in ast.walk(tree):
        if isinstance(n, ast.Import):
            out |= {a.name.split(".")[0] for a in n.names}
        elif isinstance(n, ast.ImportFrom) and n.module and n.level == 0:
            out.add(n.module.split(".")[0])
    return out


def _py_files(sub):
    d = os.path.join(ROOT, sub)
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


@pytest.mark.parametrize("sub, forbidden", [
    ("oracle", {"paper_2410_17203_gb300"}),
    ("paper_2410_17203_gb300", {"oracle"}),
    ("gridgen", {"oracle", "paper_2410_17203_gb300"}),
])
def test_no_cross_imports(sub, forbidden):
    for f in _py_files(sub):
        assert not (_imports(f) & forbidden), (f, _imports(f) & forbidden)


def test_cuda_sources_do_not_include_oracle_files():
    csrc = os.path.join(ROOT, "paper_2410_17203_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        src = open(os.path.join(csrc, f)).read()
        assert "oracle" not in src.lower(), f
