"""Every global name the committed Python code reads is defined (no GPU).

A name that a function reads but that no import, assignment or definition at module
level (or a builtin) provides only fails when that line runs; for bench.py that is on
the GPU machine, after minutes of work. The symbol tables of the compiler give the check
without running anything: a symbol a scope resolves as global must be bound at module
level.
"""
import builtins
import os
import symtable

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODULE_NAMES = {"__file__", "__name__", "__doc__", "__spec__", "__builtins__", "__loader__",
                "__package__", "__path__", "__annotations__"}


def _python_files():
    out = [os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")]
    for d in ("paper_2204_08147_gb300", "oracle", "workloads", "tests"):
        for dirpath, _, files in os.walk(os.path.join(ROOT, d)):
            if "_build" in dirpath or "__pycache__" in dirpath:
                continue
            out += [os.path.join(dirpath, f) for f in sorted(files) if f.endswith(".py")]
    return out


def _walk(table):
    yield table
    for child in table.get_children():
        yield from _walk(child)


def undefined_globals(path: str) -> list[str]:
    top = symtable.symtable(open(path).read(), path, "exec")
    bound = set(dir(builtins)) | MODULE_NAMES
    for sym in top.get_symbols():
        if sym.is_assigned() or sym.is_imported() or sym.is_namespace():
            bound.add(sym.get_name())
    # names a function declares `global` and assigns
    for t in _walk(top):
        if t is top:
            continue
        for sym in t.get_symbols():
            if sym.is_declared_global() and sym.is_assigned():
                bound.add(sym.get_name())
    missing = []
    for t in _walk(top):
        for sym in t.get_symbols():
            name = sym.get_name()
            if not sym.is_referenced() or name in bound:
                continue
            if t is top or sym.is_global():
                missing.append(f"{t.get_name()}:{name}")
    return sorted(set(missing))


@pytest.mark.parametrize("path", _python_files(), ids=lambda p: os.path.relpath(p, ROOT))
def test_no_undefined_global_names(path):
    assert undefined_globals(path) == []


def test_the_check_finds_a_missing_function(tmp_path):
    """The check itself: a call of a function that was deleted is reported."""
    p = tmp_path / "m.py"
    p.write_text("import os\n\ndef f():\n    return helper(os.sep)\n\ndef g(x):\n    return [y for y in x]\n")
    assert undefined_globals(str(p)) == ["f:helper"]
