"""Static checks of the scripts that only run in full on a GPU (bench.py,
serve.py, the entry points): they parse, and every name they read is bound
somewhere in the module (imported, assigned, a parameter or a builtin)."""
import ast
import builtins
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRIPTS = ["bench.py", "__graft_entry__.py", "paper_2507_09337_b300/serve.py", "paper_2507_09337_b300/binding.py",
           "paper_2507_09337_b300/workloads.py", "paper_2507_09337_b300/build.py"]


@pytest.mark.parametrize("path", SCRIPTS)
def test_every_read_name_is_bound(path):
    tree = ast.parse(open(os.path.join(ROOT, path)).read(), filename=path)
    bound = set(dir(builtins)) | {"__file__", "__name__"}
    for node in ast.walk(tree):
        if isinstance(node, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            bound.add(node.name)
        elif isinstance(node, ast.Name) and isinstance(node.ctx, (ast.Store, ast.Del)):
            bound.add(node.id)
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            for a in node.names:
                bound.add((a.asname or a.name).split(".")[0])
        elif isinstance(node, ast.arg):
            bound.add(node.arg)
        elif isinstance(node, ast.ExceptHandler) and node.name:
            bound.add(node.name)
    read = {n.id for n in ast.walk(tree) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
    assert not (read - bound), f"{path}: unbound names {sorted(read - bound)}"
