"""The C-ABI library builds for sm_103a, loads, and exports every function
include/liblm.h declares (no GPU needed: nothing is computed)."""
import os
import re
import subprocess

from paper_2405_15197_gb300 import build, liblm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "liblm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:lm_status|void|const char\*|long long)\s+(lm_\w+)\(", txt, re.M)))


def test_header_functions_exported():
    path = build.build()
    names = declared()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(lm_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = liblm.load()
    for n in names:
        assert getattr(lib, n) is not None
    assert set(liblm.EXPORTS) <= set(names)


def test_status_strings_and_header():
    liblm.load()
    assert liblm.lm_status_string(0) == "ok"
    assert "capacity" in liblm.lm_status_string(4)
    h = liblm.lm_stl_header(293296)
    assert len(h) == 84 and int.from_bytes(h[80:], "little") == 293296


def test_built_for_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of lm_lattice, lm_options and lm_metamesh_view have
    the size and field offsets a C compiler gives the header's structs."""
    import ctypes
    structs = {"lm_lattice": liblm.lm_lattice, "lm_options": liblm.lm_options,
               "lm_metamesh_view": liblm.lm_metamesh_view}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "liblm.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, val = ln.split()
        got[(name, field)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
