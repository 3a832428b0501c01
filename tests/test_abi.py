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


def test_struct_layouts_match_the_header(tmp_path):
    """Size and field offsets of every struct the binding mirrors, as the C compiler lays
    them out from pog.h, against the ctypes declarations."""
    structs = {"pog_options": pog.pog_options, "pog_stats_t": pog.pog_stats_t, "pog_volume": pog.pog_volume}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pog.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        struct, field, value = ln.split()
        got[(struct, field)] = int(value)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
