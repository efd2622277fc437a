"""Every name that the benchmark and the binding read is bound somewhere in their module
(CPU only): catches a misspelt or missing constant before a GPU run reaches it.
Scope-insensitive (a name bound anywhere in the file counts), so it finds names bound
nowhere, which is the failure that costs a GPU call."""
import ast
import builtins
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = ["bench.py", "__graft_entry__.py", "paper_1112_5280_gb300/lqcd.py",
         "paper_1112_5280_gb300/serve.py", "paper_1112_5280_gb300/synth.py"]


def _unbound(path):
    tree = ast.parse(open(path).read())
    bound = set(dir(builtins)) | {"__file__", "__name__"}
    for node in ast.walk(tree):
        if isinstance(node, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            bound.add(node.name)
        elif isinstance(node, ast.Name) and isinstance(node.ctx, (ast.Store, ast.Del)):
            bound.add(node.id)
        elif isinstance(node, ast.arg):
            bound.add(node.arg)
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            for a in node.names:
                bound.add((a.asname or a.name).split(".")[0])
        elif isinstance(node, ast.ExceptHandler) and node.name:
            bound.add(node.name)
        elif isinstance(node, (ast.Global, ast.Nonlocal)):
            bound.update(node.names)
    used = {n.id for n in ast.walk(tree) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
    return sorted(used - bound)


@pytest.mark.parametrize("rel", FILES)
def test_no_unbound_names(rel):
    assert _unbound(os.path.join(ROOT, rel)) == []
