"""The boundary from plain C: include/mms.h compiles as pedantic C99 (and
as C++), and a C program linked against libmms.so makes host-side calls and
gets the documented refusals -- no GPU needed."""
import os
import shutil
import subprocess

import pytest

import paper_2507_11067_gb300 as mms
from paper_2507_11067_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "_build")


@pytest.mark.parametrize("cc,std", [("gcc", ["-std=c99", "-pedantic"]), ("g++", ["-x", "c++", "-std=c++11"])])
def test_c_program_against_the_library(cc, std):
    if shutil.which(cc) is None:
        pytest.skip(f"{cc} not installed")
    mms.build()
    libdir = os.path.dirname(_lib.library_path())
    os.makedirs(OUT, exist_ok=True)
    exe = os.path.join(OUT, f"abi_from_c_{cc.replace('+', 'p')}")
    src = os.path.join(ROOT, "tests", "c", "abi_from_c.c")
    cmd = [cc] + std + ["-Wall", "-Wextra", "-Werror", "-I" + os.path.join(ROOT, "include"), src,
                        "-L" + libdir, "-lmms", "-Wl,-rpath," + libdir, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
