"""The C-ABI library builds, loads, and exports every symbol that include/pog.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2601_17026_gb300 import build as build_mod
from paper_2601_17026_gb300 import pog

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pog.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"POG_API\s+[\w\s\*]+?\b(pog_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    return build_mod.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pog_build", "pog_maxflow", "pog_surface", "pog_free", "pog_strerror"):
        assert required in names
    assert sorted(pog.EXPORTED) == sorted(names), "binding and header disagree"


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pog_\w+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, f"not exported: {missing}"


def test_library_loads_and_strerror(lib_path):
    lib = pog.load(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name)
    assert pog.pog_strerror(0) == "ok"
    assert "int32" in pog.pog_strerror(pog.POG_E_OVERFLOW)
    assert pog.pog_strerror(999) == "unknown status"


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "use.c"
    src.write_text('#include "pog.h"\nint main(void) { return (int)POG_OK + (int)sizeof(pog_stats_t) % 1; }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), "-c", str(src), "-o",
                    str(tmp_path / "use.o")], check=True)


def test_options_struct_layout():
    assert ctypes.sizeof(pog.pog_options) == 32
    assert ctypes.sizeof(pog.pog_stats_t) == 112
