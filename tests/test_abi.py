"""Host-side checks of the C ABI: the library builds, loads and exports every
entry point declared in include/iga.h (no GPU calls)."""
import ctypes
import os
import re
import shutil
import subprocess

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
    assert L.iga_kron_apply(None, None, 0, 1.0, None, 0.0, None, 0) == 1
    assert L.iga_last_error(None) == b"null context"
    assert L.iga_launch_count(None) == 0


def test_header_cites_the_paper():
    hdr = open(os.path.join(ROOT, "include", "iga.h")).read()
    for needle in ("KKT_red", "KKTSystem", "massMatrix1D", "eq. tt", "geometryMapping"):
        assert needle in hdr, needle


# public structs of include/iga.h and their ctypes mirrors in the binding
_STRUCTS = {"iga_geometry": "Geometry_", "iga_space": "Space_", "iga_target": "Target_",
            "iga_solve_opts": "SolveOpts_", "iga_solve_info": "SolveInfo_"}


def _c_layouts(tmp_path):
    """sizeof and every field offset of the public structs, as a C compiler
    lays them out from the header (host gcc, no CUDA)."""
    from paper_1811_06797_gb300 import iga
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "iga.h"', "int main(void) {"]
    for cname, pyname in _STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in getattr(iga, pyname)._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no host C compiler")
def test_binding_struct_layouts_match_header(tmp_path):
    """Every ctypes structure of the binding has the C layout of the header:
    same size and the same offset for every field (a field added on one side
    only shifts the ones after it)."""
    from paper_1811_06797_gb300 import iga
    c = _c_layouts(tmp_path)
    for cname, pyname in _STRUCTS.items():
        py = getattr(iga, pyname)
        assert ctypes.sizeof(py) == c[(cname, "size")], cname
        for field, _ in py._fields_:
            assert getattr(py, field).offset == c[(cname, field)], (cname, field)
