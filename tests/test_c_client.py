"""The C ABI from C99 programs: include/lbm.h compiles as plain C (no C++) with warnings as errors;
one program calls the entry points that need no GPU, another (GPU) runs a droplet end to end."""
import os
import shutil
import subprocess

import pytest

from paper_2306_16274_gb300 import lbm as L

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _build_and_run(tmp_path, name):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    L.lib()                                   # builds nothing; fails loudly if the library is missing
    libdir = os.path.dirname(L.LIB_PATH)
    exe = str(tmp_path / name)
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "c", name + ".c"), "-o", exe, "-L", libdir, "-llbm", "-lm", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_c99_client(tmp_path):
    _build_and_run(tmp_path, "abi_host")


@pytest.mark.gpu
def test_c99_client_runs_a_simulation(tmp_path):
    # the whole path through the C ABI with host pointers, no Python in between
    import __graft_entry__
    __graft_entry__.build()
    _build_and_run(tmp_path, "abi_gpu")
