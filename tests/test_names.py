"""Every global name a function of the package, the bench or the oracle
reads is bound at module level (a scope-aware check with ``symtable``):
catches code paths that only run on a GPU reading a name that no longer
exists."""
import builtins
import glob
import os
import symtable

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(glob.glob(os.path.join(ROOT, "paper_2507_11067_gb300", "*.py"))
               + glob.glob(os.path.join(ROOT, "oracle", "*.py"))
               + glob.glob(os.path.join(ROOT, "workloads", "*.py"))
               + glob.glob(os.path.join(ROOT, "tests", "*.py"))
               + [os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")])


def _unbound(path):
    with open(path) as f:
        top = symtable.symtable(f.read(), path, "exec")
    bound = {s.get_name() for s in top.get_symbols()
             if s.is_assigned() or s.is_imported() or s.is_namespace()}
    bound |= set(dir(builtins)) | {"__file__"}
    bad = []

    def walk(t):
        for c in t.get_children():
            for s in c.get_symbols():
                if (s.is_referenced() and s.is_global() and not s.is_declared_global()
                        and s.get_name() not in bound):
                    bad.append((c.get_name(), c.get_lineno(), s.get_name()))
            walk(c)
    walk(top)
    return bad


@pytest.mark.parametrize("path", FILES, ids=lambda p: os.path.relpath(p, ROOT))
def test_functions_read_only_bound_globals(path):
    assert _unbound(path) == []
