"""Host-side checks of the C ABI: the library builds, loads and exports every
entry point declared in include/iga.h (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "iga.h")).read()
    return sorted(set(re.findall(r"\b(iga_[a-z0-9_]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1811_06797_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name


def test_binding_covers_header(libpath):
    from paper_1811_06797_gb300 import iga
    assert iga.exported_symbols() == _declared()
    iga.lib()   # every signature resolves


def test_null_context_is_rejected(libpath):
    from paper_1811_06797_gb300 import iga
    L = iga.lib()
    assert L.iga_kron_apply(None, None, 1.0, None, 0.0, None, 0) == 1
    assert L.iga_last_error(None) == b"null context"
    assert L.iga_launch_count(None) == 0


def test_header_cites_the_paper():
    hdr = open(os.path.join(ROOT, "include", "iga.h")).read()
    for needle in ("KKT_red", "KKTSystem", "massMatrix1D", "eq. tt", "geometryMapping"):
        assert needle in hdr, needle
