"""The C ABI library builds, loads and exports every function include/muca.h declares
(no compute: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(muca_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("muca_init", "muca_iterate", "muca_merge_and_update", "muca_get_lnW", "muca_get_histogram",
              "muca_get_reweight", "muca_get_state", "muca_set_state", "muca_free"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1312_2213_gb300 as m

    lib = m.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding carries the same names
    assert not [n for n in declared_functions() if not hasattr(m, n)]


def test_workspace_size_and_argument_errors_without_gpu():
    import paper_1312_2213_gb300 as m

    n = m.muca_workspace_size(m.ISING2D, 32, 2, 8192)
    assert n >= 8192 * 32 * 4
    with pytest.raises(m.MucaError) as e:
        m.muca_workspace_size(m.ISING2D, 30, 2, 64)   # unsupported L
    assert e.value.code == -1
    with pytest.raises(m.MucaError):
        m.muca_workspace_size(m.POTTS2D, 32, 17, 64)  # q > 16
    with pytest.raises(m.MucaError):
        m.muca_workspace_size(m.ISING2D, 32, 2, 0)    # p < 1
    assert "p must be" in m.muca_last_error()
