"""The C ABI library builds for sm_103a, loads without a GPU and exports every entry point
include/ivis.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", hdr)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ivis_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_all_declared_symbols():
    from paper_2609_17636_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert "ivis_cost_grad" in declared and "ivis_solve" in declared
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2609_17636_b300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()


def test_missing_library_fails_loudly(tmp_path):
    from paper_2609_17636_b300 import _lib
    saved = _lib._LIB
    try:
        _lib._LIB = None
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._LIB = saved


def test_plan_rejects_bad_config_without_gpu():
    """Argument validation happens on the host before any device call."""
    from paper_2609_17636_b300 import _lib
    L = _lib.load()
    cfg = _lib.Config(64, 1, 1, 48, 1e-5, 0, 1e-9, 0, 0.0, 0.0, 1, 0, 0, 0, 0)  # nb not a power of two
    p = ctypes.c_void_p()
    st = L.ivis_plan(ctypes.byref(cfg), None, ctypes.byref(p))
    assert st == 1 and not p.value
    assert b"power of two" in L.ivis_last_error(None)


def test_rayleigh_jeans_entry_point_matches_the_oracle():
    """A host-only entry point: callable without a GPU."""
    import oracle
    from paper_2609_17636_b300 import rayleigh_jeans
    for f in (1.0e8, 1.4204058e9, 2.3e10):
        assert abs(rayleigh_jeans(f) - oracle.rayleigh_jeans_factor(f)) <= 1e-14 * oracle.rayleigh_jeans_factor(f)
