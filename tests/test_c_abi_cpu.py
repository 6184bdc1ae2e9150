"""The ABI from plain C: tests/c_abi_host.c is compiled with gcc against
include/xyl.h, linked to the in-tree libxyl.so and run (host calls only, no
GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_uses_the_abi(tmp_path):
    from paper_1211_3991_gb300 import build
    lib = build.build()
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    exe = str(tmp_path / "c_abi_host")
    libdir = os.path.dirname(lib)
    subprocess.run([gcc, "-std=c11", "-O1", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_host.c"), "-o", exe, "-L", libdir, "-l:libxyl.so",
                    f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")
    assert r.stdout.count("workspace") == 3
