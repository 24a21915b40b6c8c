"""The C-ABI library builds, loads and exports every function declared in
include/tdbem.h (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tdbem_\w+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2505_00715_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_2505_00715_gb300 import _lib
    assert set(_declared()) <= set(_lib.EXPORTS)


def test_product_path_fails_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2505_00715_gb300 as td
    with pytest.raises(td.TdbemError):
        td.Context(0)
