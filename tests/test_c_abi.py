"""The boundary from plain C: include/mms.h compiles as pedantic C99 (and
as C++), and a C program linked against libmms.so makes host-side calls and
gets the documented refusals -- no GPU needed.  On a GPU the same program
checks that AUTO follows the library's built-in tuned table, which build.py
compiles in from tuned.json (the rows load_table() would register)."""
import json
import os
import shutil
import subprocess

import pytest

import paper_2507_11067_gb300 as mms
from paper_2507_11067_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "_build")


def _compile(cc, std):
    mms.build()
    libdir = os.path.dirname(_lib.library_path())
    os.makedirs(OUT, exist_ok=True)
    exe = os.path.join(OUT, f"abi_from_c_{cc.replace('+', 'p')}")
    src = os.path.join(ROOT, "tests", "c", "abi_from_c.c")
    cmd = [cc] + std + ["-Wall", "-Wextra", "-Werror", "-I" + os.path.join(ROOT, "include"), src,
                        "-L" + libdir, "-lmms", "-Wl,-rpath," + libdir, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


@pytest.mark.parametrize("cc,std", [("gcc", ["-std=c99", "-pedantic"]), ("g++", ["-x", "c++", "-std=c++11"])])
def test_c_program_against_the_library(cc, std):
    if shutil.which(cc) is None:
        pytest.skip(f"{cc} not installed")
    exe = _compile(cc, std)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_built_in_table_is_the_registered_rows(tmp_path):
    # the rows build.py compiles in are, per GPU and (shape, r, path), the
    # variant of the largest tuned grid -- what tune.load_table() registers
    import importlib
    b = importlib.import_module("paper_2507_11067_gb300.build")
    table = tmp_path / "t.json"
    table.write_text(json.dumps({
        "G1|box|r2|bf16x3|512x512x512": {"variant": 3, "ms": []},
        "G1|box|r2|bf16x3|64x64x64": {"variant": 1, "ms": []},
        "G1|star|r4|cuda_core|1024x1024x1024": {"variant": 12, "ms": []},
        "G2|box2d|r3|cuda_core|8192x8192x1": {"variant": 5, "ms": []}}))
    assert b.tuned_rows(str(table)) == [("G1", 0, 4, 1, 12), ("G1", 1, 2, 4, 3), ("G2", 3, 3, 1, 5)]
    inc = open(b.write_tuned_defaults(str(table), str(tmp_path / "gen"))).read()
    for row in ('{"G1", 0, 4, 1, 12}', '{"G1", 1, 2, 4, 3}', '{"G2", 3, 3, 1, 5}'):
        assert row in inc
    # the library's own copy is generated from the committed table
    committed = open(os.path.join(b.GEN, "tuned_defaults.inc")).read()
    for gpu, shape, r, path, var in b.tuned_rows():
        assert f'{{"{gpu}", {shape}, {r}, {path}, {var}}}' in committed


@pytest.mark.gpu
def test_c_program_sees_the_built_in_table_on_the_gpu():
    torch = pytest.importorskip("torch")
    import importlib
    b = importlib.import_module("paper_2507_11067_gb300.build")
    name = torch.cuda.get_device_name(0)
    rows = {(s, r, p): v for g, s, r, p, v in b.tuned_rows() if g == name}
    box, bf16x3, cuda_core = 1, 4, 1
    path = bf16x3 if (box, 2, bf16x3) in rows else cuda_core
    variant = rows.get((box, 2, path), 0)
    exe = _compile("gcc", ["-std=c99", "-pedantic"])
    r = subprocess.run([exe, "gpu", str(path), str(variant)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
    print(f"{name}: AUTO of box r=2 from C = path {path}, variant {variant}")
