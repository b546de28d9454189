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


def _dummy(argtype):
    """A harmless value of a prototype's argument type (null pointers, zero sizes)."""
    if argtype in (ctypes.c_void_p, ctypes.c_char_p):
        return None
    if isinstance(argtype, type) and issubclass(argtype, ctypes._Pointer):
        return None
    return argtype(0)


def test_null_handles_are_refused_without_gpu():
    """Every entry point that takes a context or batch handle refuses a NULL one with MUCA_ERR_ARG
    (and an error text) before touching the device; the free functions accept NULL."""
    import paper_1312_2213_gb300 as m
    from paper_1312_2213_gb300 import _native

    lib = m.load()
    skip = {"muca_last_error", "muca_init", "muca_init_ex", "muca_workspace_size", "muca_det_math",
            "muca_free", "muca_batch_free"}
    checked = []
    for name, (res, args) in _native.PROTOTYPES.items():
        if name in skip or not args or args[0] is not ctypes.c_void_p:
            continue
        fn = getattr(lib, name)
        vals = [None] + [_dummy(a) for a in args[1:]]
        if name == "muca_set_param":
            vals[1] = b"flat_ratio"
        rc = fn(*vals)
        assert rc == -1, (name, rc)
        assert m.muca_last_error(), name
        checked.append(name)
    assert len(checked) >= 25
    assert lib.muca_free(None) == 0 and lib.muca_batch_free(None) == 0


def test_init_refuses_bad_configurations_without_gpu():
    """muca_init / muca_init_ex validate the configuration, and an arena's size and alignment,
    before any device call; the output handle is left NULL."""
    from paper_1312_2213_gb300 import _native

    lib = _native.load()
    h = ctypes.c_void_p(1234)
    for system, L, q, p in ((0, 30, 2, 64), (1, 32, 17, 64), (1, 32, 1, 64), (0, 32, 2, 0), (3, 1, 0, 64),
                            (3, 129, 0, 64), (9, 32, 2, 64)):
        assert lib.muca_init(ctypes.byref(h), system, L, q, p, 1) == -1, (system, L, q, p)
        assert h.value is None
    assert lib.muca_init(None, 0, 32, 2, 64, 1) == -1
    need = ctypes.c_size_t()
    assert lib.muca_workspace_size(0, 32, 2, 64, ctypes.byref(need)) == 0
    # a NULL arena, one too small, one off the 256-byte alignment: refused, never dereferenced
    assert lib.muca_init_ex(ctypes.byref(h), 0, 32, 2, 64, 1, None, need.value) == -1
    assert lib.muca_init_ex(ctypes.byref(h), 0, 32, 2, 64, 1, ctypes.c_void_p(1 << 20), need.value - 1) == -3
    assert lib.muca_init_ex(ctypes.byref(h), 0, 32, 2, 64, 1, ctypes.c_void_p((1 << 20) + 16), need.value) == -3
    assert b"aligned" in lib.muca_last_error()
    assert h.value is None
    # det_math validates its selector first
    assert lib.muca_det_math(2, None, None, 0) == -1
