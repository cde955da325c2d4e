"""include/dfdm.h is a plain C interface: a C program (tests/c/abi_check.c)
compiles with gcc against the header alone, links libdfdm.so and makes the
calls that need no GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_plain_c_program_uses_the_library(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2004_14229_gb300._build import build_library
    lib = build_library()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "abi_check")
    cmd = ["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "c", "abi_check.c"), "-o", exe, "-L", libdir, "-ldfdm",
           "-Wl,-rpath," + libdir, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "FAIL" not in r.stdout
