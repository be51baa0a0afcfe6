"""The oracle and the CUDA path share no code: no module of the product package
imports the oracle, the oracle imports nothing of the product package, and the
input generators (workloads/) import neither (they hold none of the method's
arithmetic).  Checked on the import statements of every source file."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out


def _py_files(pkg):
    d = os.path.join(ROOT, pkg)
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


@pytest.mark.parametrize("pkg,forbidden", [
    ("paper_2101_05917_gb300", {"oracle"}),
    ("oracle", {"paper_2101_05917_gb300"}),
    ("workloads", {"oracle", "paper_2101_05917_gb300"}),
])
def test_no_shared_code(pkg, forbidden):
    files = _py_files(pkg)
    assert files
    for f in files:
        bad = _imports(f) & forbidden
        assert not bad, (f, bad)


def test_native_sources_do_not_reference_the_oracle():
    csrc = os.path.join(ROOT, "paper_2101_05917_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower(), f
