"""The C-ABI library builds, loads and exports every symbol include/mortar.h declares.

No compute call is made (these run without a GPU).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2202_03933_gb300 import build, _native
    build()
    return _native


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "mortar.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mortar_[a-z_0-9]+)\s*\(", txt)))


def test_header_and_binding_agree(native):
    decl = declared_functions()
    assert len(decl) >= 20
    assert sorted(native.EXPORTS) == decl


def test_library_exports_every_declared_symbol(native):
    L = native.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_host_only_calls(native):
    L = native.lib()
    o = native.Options()
    assert L.mortar_default_options(ctypes.byref(o)) == 0
    assert o.newton_max_iter == 20 and o.newton_tol == 1e-14 and o.search_inflation == 1e-9
    assert o.clip_tol_rel == 1e-12 and o.merge_tol_rel == 1e-10 and o.area_tol_rel == 1e-14
    assert o.bin_margin == 0.0 and o.integration == 0 and o.element_rule_n == 8 and o.facing_test == 0
    assert L.mortar_default_options(None) == -1
    assert L.mortar_status_string(-4) == b"MORTAR_ERR_CAPACITY"
    assert L.mortar_status_string(0) == b"MORTAR_OK"
    L.mortar_destroy(None)   # NULL is ignored


def test_product_path_fails_loudly_without_library(monkeypatch):
    from paper_2202_03933_gb300 import _native
    monkeypatch.setattr(_native, "LIB_PATH", "/nonexistent/libmortar_gb300.so")
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _native.lib()


def test_package_does_not_import_oracle():
    import subprocess
    import sys
    code = ("import sys; import paper_2202_03933_gb300.mortar, paper_2202_03933_gb300.inputs; "
            "assert 'oracle' not in sys.modules, 'product imported the oracle'")
    subprocess.run([sys.executable, "-c", code], check=True, cwd=ROOT)
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2202_03933_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "mortar_oracle" not in src, f
