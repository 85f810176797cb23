"""Every name a function of bench.py (and of the package's Python modules) reads
is bound somewhere it can see: its own scope, an enclosing function, the module
or the builtins.  A measurement the driver runs once per round must not stop on
a NameError in a path the CPU tests do not execute."""
import ast
import builtins
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = ["bench.py", "__graft_entry__.py", os.path.join("paper_1803_03922_gb300", "__init__.py"),
         os.path.join("paper_1803_03922_gb300", "autotune.py"), os.path.join("paper_1803_03922_gb300", "_build.py")]


def _bound(node):
    """Names bound directly in the scope of `node` (a module, function or lambda)."""
    out = set()
    if isinstance(node, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda)):
        a = node.args
        for x in a.posonlyargs + a.args + a.kwonlyargs:
            out.add(x.arg)
        if a.vararg:
            out.add(a.vararg.arg)
        if a.kwarg:
            out.add(a.kwarg.arg)
    body = node.body if isinstance(node.body, list) else [node.body]
    stack = list(body)
    while stack:
        n = stack.pop()
        if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            out.add(n.name)
            continue  # its body is its own scope
        if isinstance(n, ast.Lambda):
            continue
        if isinstance(n, (ast.Import, ast.ImportFrom)):
            for al in n.names:
                out.add((al.asname or al.name).split(".")[0])
        elif isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            out.add(n.id)
        elif isinstance(n, (ast.Global, ast.Nonlocal)):
            out.update(n.names)
        elif isinstance(n, ast.ExceptHandler) and n.name:
            out.add(n.name)
        elif isinstance(n, ast.arg):
            out.add(n.arg)
        stack.extend(ast.iter_child_nodes(n))
    return out


def _loads(node):
    """Names read in the scope of `node`, not descending into nested scopes."""
    out = []
    body = node.body if isinstance(node.body, list) else [node.body]
    stack = list(body)
    if isinstance(node, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda)):
        stack += node.args.defaults + [d for d in node.args.kw_defaults if d is not None]
    while stack:
        n = stack.pop()
        if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda, ast.ClassDef)):
            continue
        if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load):
            out.append(n)
        stack.extend(ast.iter_child_nodes(n))
    return out


def _unbound(path):
    tree = ast.parse(open(path).read(), path)
    missing = []
    comp_names = set()
    for n in ast.walk(tree):  # comprehension targets live in their own scope; accept them everywhere
        if isinstance(n, ast.comprehension):
            for t in ast.walk(n.target):
                if isinstance(t, ast.Name):
                    comp_names.add(t.id)

    def visit(node, visible):
        here = visible | _bound(node)
        if not isinstance(node, ast.Module):
            for name in _loads(node):
                if name.id not in here and name.id not in comp_names and not hasattr(builtins, name.id):
                    missing.append("%s:%d %s" % (os.path.basename(path), name.lineno, name.id))
        for child in ast.walk(node):
            if child is node:
                continue
            if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda)) and _parent_scope(tree, child) is node:
                visit(child, here)

    visit(tree, set())
    return missing


def _parent_scope(tree, target):
    """The innermost function or module whose scope contains `target`."""
    best = tree
    for n in ast.walk(tree):
        if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda, ast.ClassDef)) and n is not target:
            for c in ast.walk(n):
                if c is target:
                    if best is tree or _contains(best, n):
                        best = n
    return best if not isinstance(best, ast.ClassDef) else tree


def _contains(outer, inner):
    return any(c is inner for c in ast.walk(outer))


@pytest.mark.parametrize("rel", FILES)
def test_functions_read_only_bound_names(rel):
    assert _unbound(os.path.join(ROOT, rel)) == []
