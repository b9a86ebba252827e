"""The C ABI from C: every public header compiles as C (gcc, -std=c99
-Wall -Werror) and a C client calls the host-side entry points of the built
libraries (planning, sizes, plan export, error reporting) without a GPU."""
import os
import shutil
import subprocess

import pytest

from paper_2509_21037_gb300 import _build, _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client_of_the_abi(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    _native.sc_lib()                      # the libraries are built (fails loudly otherwise)
    cuda = _build._cuda_home()
    lib = _native.LIBDIR
    exe = str(tmp_path / "c_abi_check")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_check.c"), "-o", exe, "-L", lib, "-lsc", "-lscfactor",
           "-Wl,-rpath," + lib, "-L", os.path.join(cuda, "lib64"), "-Wl,-rpath," + os.path.join(cuda, "lib64"),
           "-lcudart", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "C ABI OK" in r.stdout
