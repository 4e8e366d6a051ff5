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
