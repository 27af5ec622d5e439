"""The C-ABI library builds, loads without a GPU, and exports every entry point declared in
include/*.h (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mgm_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2204_06154_gb300.build import build
    path = build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 18
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_2204_06154_gb300 import mgm
    assert set(mgm.EXPORTS) == _declared()


def test_status_strings_without_gpu():
    from paper_2204_06154_gb300 import mgm
    L = mgm.lib()
    for code, name in mgm.STATUS.items():
        assert L.mgm_status_string(code).decode() == name
