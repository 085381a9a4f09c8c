"""The C ABI from a C99 program: include/lbm.h compiles as plain C (no C++) with warnings as
errors, and a program linked against liblbm.so calls the entry points that need no GPU."""
import os
import shutil
import subprocess

import pytest

from paper_2306_16274_gb300 import lbm as L

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_c99_client(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    L.lib()                                   # builds nothing; fails loudly if the library is missing
    libdir = os.path.dirname(L.LIB_PATH)
    exe = str(tmp_path / "abi_host")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "c", "abi_host.c"), "-o", exe, "-L", libdir, "-llbm", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
