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
