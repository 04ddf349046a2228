"""The boundary as a C user sees it: include/ifmm.h compiles as C99, a C program
links against libifmm.so by name, resolves every declared entry point, and runs
the host-side tree and coloring calls and the error protocol (no GPU needed)."""

import os
import re
import shutil
import subprocess

import pytest

from paper_1905_10602_gb300 import build as _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ifmm.h")
SRC = os.path.join(ROOT, "tests", "c_abi_check.c")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_program_links_and_runs(tmp_path):
    lib = _build.build()
    names = re.findall(r"^\s*(?:ifmm_status|void|const char\*)\s+(\w+)\s*\(", open(HEADER).read(), re.M)
    assert len(names) > 20
    (tmp_path / "abi_table.h").write_text("#define IFMM_ABI_TABLE " + " ".join(f"X({n})" for n in names) + "\n")
    exe = str(tmp_path / "c_abi_check")
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-include", str(tmp_path / "abi_table.h"),
           "-I", os.path.join(ROOT, "include"), SRC, "-o", exe, "-L" + libdir, "-lifmm", "-Wl,-rpath," + libdir, "-lm"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "c_abi ok" in r.stdout, r.stdout + r.stderr
