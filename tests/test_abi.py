"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/*.h declares (no compute calls)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(amg_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2011_13325_gb300 import amg, build
    if not os.path.exists(amg.LIBPATH):
        build.build()
    return amg


def test_header_declares_entry_points():
    names = _declared()
    for n in ("amg_upload_hierarchy", "amg_galerkin", "amg_vcycle", "amg_pcg_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    L = ctypes.CDLL(lib.LIBPATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    # the Python binding marshals exactly these entry points
    assert set(lib.exported_symbols()) <= set(_declared())


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2011_13325_gb300 import amg
    monkeypatch.setattr(amg, "LIBPATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(amg, "_lib", None)
    with pytest.raises(RuntimeError):
        amg.lib()
