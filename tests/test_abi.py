"""The C-ABI library builds, loads and exports every symbol include/krylov.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "krylov.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2104_01253_gb300 import build as b
    if not os.path.exists(b.LIB) or any(os.path.getmtime(s) > os.path.getmtime(b.LIB)
                                        for s in b.sources()):
        b.build()
    return b.LIB


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("dcgs2_arnoldi_step", "gmres_solve", "krylov_schur_eigs", "kc_create"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_names_match(lib_path):
    from paper_2104_01253_gb300 import _lib
    lib = _lib.load(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name)
    assert set(_lib.exported_names()) <= set(declared_functions())


STRUCTS = ("kc_csr", "kc_arnoldi", "kc_gmres_opts", "kc_gmres_info", "kc_ks_opts")


def test_ctypes_structs_match_the_header(tmp_path):
    """sizeof and every field offset of the header's structs, as the C compiler lays them
    out, equal those of the binding's ctypes mirrors."""
    from paper_2104_01253_gb300 import _lib
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "krylov.h"', 'int main(void) {']
    for name in STRUCTS:
        cls = getattr(_lib, name)
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    import ctypes
    for name in STRUCTS:
        cls = getattr(_lib, name)
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)
