"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and exports every
symbol include/blcoc.h declares.  No compute call is made here (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(blcoc_[a-z_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1601_05362_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ("blcoc_create", "blcoc_solve", "blcoc_get_info", "blcoc_destroy", "blcoc_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(blcoc_[a-z_]+)\b", out))
    missing = _declared_symbols() - exported
    assert not missing, missing


def test_binding_loads_and_binds_all_symbols(libpath):
    from paper_1601_05362_gb300 import blcoc
    lib = blcoc.load_library()
    assert set(blcoc.SIGNATURES) == _declared_symbols()
    for name in blcoc.SIGNATURES:
        assert hasattr(lib, name)
    # status strings need no device
    assert blcoc.status_string(0) == "BLCOC_OK"
    assert blcoc.status_string(6) == "BLCOC_BREAKDOWN"


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1601_05362_gb300 import blcoc
    with pytest.raises(RuntimeError, match="not built"):
        blcoc._lib, saved = None, blcoc._lib
        try:
            blcoc.load_library(str(tmp_path / "missing.so"))
        finally:
            blcoc._lib = saved


def test_binding_rejects_lazy_conjugate_views():
    """The C ABI reads raw memory; a torch conj()/neg view does not hold its values there."""
    torch = pytest.importorskip("torch")
    from paper_1601_05362_gb300 import blcoc
    x = torch.zeros((4, 2), dtype=torch.complex128)
    with pytest.raises(ValueError, match="lazy conj"):
        blcoc._ptr(x.conj())
    blcoc._ptr(x.conj_physical())
