"""mms_stencil_apply_noalloc: the tensor-core star sweep whose temporary grid
is the library's fixed device array instead of a per-call allocation.

The GPU test makes two calls in a row (the second on a smaller grid with
other data and weights, so stale contents of the shared array from the first
call would show) and compares each with mms_stencil_apply_ex on the same
path and variant.  The CPU tests check that the entry point refuses what it
cannot do before it touches the device.
"""
import ctypes

import numpy as np
import pytest

import paper_2507_11067_gb300 as mms
from paper_2507_11067_gb300 import _lib
import workloads

TOL = 1e-5  # the split-precision tensor-core bar of the parity tests


@pytest.fixture(scope="module")
def lib():
    mms.build()
    return mms.load()


def _desc(c, **kw):
    return _lib.StencilDesc(kw.get("shape", 0), kw.get("radius", 4), c.ctypes.data, kw.get("nx", 8),
                            kw.get("ny", 8), kw.get("nz", 8), 0, 0, 0, 0, kw.get("path", 4), -1)


@pytest.mark.parametrize("kw,status", [
    (dict(nx=256, ny=256, nz=129), 1),      # one plane above the limit
    (dict(nx=4096, ny=4096, nz=1), 1),      # 2x the limit
    (dict(nx=(1 << 30) - 1, ny=(1 << 30) - 1, nz=(1 << 30) - 1), 1),   # a product beyond 64 bits
    (dict(shape=1), 2),                     # box: needs no temporary grid
    (dict(path=1), 2),                      # CUDA-core path
    (dict(path=5), 2),                      # naive path
    (dict(radius=5), 1),
])
def test_noalloc_refuses_before_touching_the_device(lib, kw, status):
    c = np.ones(27, np.float32)
    d = _desc(c, **kw)
    buf_in, buf_out = ctypes.create_string_buffer(64), ctypes.create_string_buffer(64)
    st = lib.mms_stencil_apply_noalloc(ctypes.byref(d), buf_in, buf_out, None)
    assert st == status, lib.mms_last_error()
    msg = lib.mms_last_error().decode()
    if status == 1 and kw.get("nx", 0) >= 256:
        assert "no-alloc limit" in msg and str(_lib.NOALLOC_MAX_POINTS) in msg


def test_noalloc_empty_interior_is_a_no_op(lib):
    c = np.ones(27, np.float32)
    d = _desc(c, nx=0)
    assert lib.mms_stencil_apply_noalloc(ctypes.byref(d), None, None, None) == 0


def _rel(a, b):
    return (a - b).abs().max().item() / max(b.abs().max().item(), 1e-30)


@pytest.mark.gpu
@pytest.mark.parametrize("path", ["bf16x3", "3xtf32"])
@pytest.mark.parametrize("r", [1, 2, 4])
def test_noalloc_matches_apply_ex_on_two_calls_in_a_row(lib, path, r):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    # first call: the largest interior the array holds; second: a small
    # ragged grid with other data and weights
    sizes = [(256, 256, _lib.NOALLOC_MAX_POINTS // (256 * 256)), (53, 41, 19)]
    assert sizes[0][0] * sizes[0][1] * sizes[0][2] == _lib.NOALLOC_MAX_POINTS
    for k, n in enumerate(sizes):
        grid = workloads.uniform_grid(*n, r, workload=3, salt=700 + 10 * r + k)
        c = workloads.normal_coeffs("star", r, workload=3, salt=700 + 10 * r + k)
        inp = mms.to_padded_device(grid, r)
        ref = mms.apply("star", r, c, inp, path=path)
        out = torch.full_like(ref, float("nan"))
        _lib.apply_noalloc(r, c, inp, out, path=path)
        torch.cuda.synchronize()
        mms.check_device()
        err = _rel(out, ref)
        print(f"star r={r} {path} n={n} call {k + 1}: no-alloc vs apply_ex max-rel {err:.3e}")
        assert torch.isfinite(out).all()
        assert err <= TOL, (n, err)
