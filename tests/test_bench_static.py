"""bench.py and the package's Python modules: every name a function reads is defined somewhere it can
see (a local, an enclosing scope, the module or the builtins), so that a path the CPU suite cannot run
(the GPU bench legs) does not fail on a typo."""
import builtins
import os
import symtable

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = ["bench.py", "__graft_entry__.py"] + [
    os.path.join("paper_2111_02912_gb300", f) for f in sorted(os.listdir(os.path.join(ROOT, "paper_2111_02912_gb300")))
    if f.endswith(".py")]


def _undefined(path):
    src = open(os.path.join(ROOT, path)).read()
    top = symtable.symtable(src, path, "exec")
    module_names = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    known = module_names | set(dir(builtins)) | {"__file__", "__name__"}
    bad = []

    def walk(tab):
        for s in tab.get_symbols():
            if s.is_referenced() and s.is_global() and not s.is_declared_global() and s.get_name() not in known:
                bad.append("%s: %s" % (tab.get_name(), s.get_name()))
        for child in tab.get_children():
            walk(child)

    for child in top.get_children():
        walk(child)
    return bad


@pytest.mark.parametrize("path", FILES)
def test_every_name_read_is_defined(path):
    assert _undefined(path) == []


def test_config_picks_counts_every_candidate_shape():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from paper_2111_02912_gb300.batch import CONFIG_CANDIDATES_2D
    picks = bench.config_picks(list(CONFIG_CANDIDATES_2D) + [CONFIG_CANDIDATES_2D[0], None])
    assert sum(picks.values()) == len(CONFIG_CANDIDATES_2D) + 2
    assert picks[",".join(str(f) for f in CONFIG_CANDIDATES_2D[0])] == 2 and picks["default"] == 1
