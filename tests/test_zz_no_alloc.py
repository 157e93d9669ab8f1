"""mms_stencil_apply_noalloc: the tensor-core star sweep whose temporary grid
is the library's fixed device array instead of a per-call allocation.

The GPU tests make two calls in a row (the second on a smaller grid with
other data and weights, so stale contents of the shared array from the first
call would show) and compare each with mms_stencil_apply_ex on the same path
and with the FP64 oracle; and they read the device's default memory pool
around a call: the two-pass form through mms_stencil_apply_ex raises its
high-water mark by the temporary grid, the no-alloc call does not raise it at
all.  The CPU tests check that the entry point refuses what it cannot do
before it touches the device.
"""
import ctypes

import numpy as np
import pytest

import oracle
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
    (dict(path=99), 1),                     # no such path
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
@pytest.mark.parametrize("r", [1, 2, 3, 4])
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
        # and against the FP64 oracle (every point of the small grid, sampled
        # points of the large one)
        if k == 1:
            o = oracle.stencil("star", r, c, grid)
            got = out.cpu().numpy().astype(np.float64)
        else:
            pts = workloads.sample_points(*n, 2000, workload=3, salt=r)
            o = oracle.stencil_points("star", r, c, grid, pts)
            got = out[pts[:, 2], pts[:, 1], pts[:, 0]].cpu().numpy().astype(np.float64)
        err = float(np.abs(got - o).max() / np.abs(o).max())
        print(f"star r={r} {path} n={n} call {k + 1}: no-alloc vs oracle max-rel {err:.3e}")
        assert err <= TOL, (n, err)


@pytest.mark.gpu
def test_noalloc_takes_nothing_from_the_memory_pool(lib):
    # The driver's default memory pool of the device (where the stream-ordered
    # allocations of mms_stencil_apply_ex come from): its used-memory
    # high-water mark, reset before a call, rises by the temporary grid in the
    # two-pass form through mms_stencil_apply_ex and not at all through the
    # no-alloc entry point.
    torch = pytest.importorskip("torch")
    cu = ctypes.CDLL("libcuda.so.1")
    dev = torch.cuda.current_device()
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), ctypes.c_int(dev)) == 0
    USED_CURRENT, USED_HIGH = 7, 8     # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH

    def attr(a):
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, ctypes.c_int(a), ctypes.byref(v)) == 0
        return v.value

    def reset_high():
        z = ctypes.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, ctypes.c_int(USED_HIGH), ctypes.byref(z)) == 0
        return attr(USED_CURRENT)

    r, n = 2, (96, 80, 40)
    grid = workloads.uniform_grid(*n, r, workload=3, salt=9)
    c = workloads.normal_coeffs("star", r, workload=3, salt=9)
    inp = mms.to_padded_device(grid, r)
    out = torch.empty((n[2], n[1], n[0]), device="cuda")
    _lib.apply_noalloc(r, c, inp, out, path="bf16x3")   # the set-up call on this device
    torch.cuda.synchronize()
    two_pass = mms.num_variants("star", r, "bf16x3") // 2   # the star's two-pass variants come second
    used = reset_high()
    mms.apply("star", r, c, inp, out, path="bf16x3", variant=two_pass)
    torch.cuda.synchronize()
    grew = attr(USED_HIGH) - used
    print(f"default pool high-water mark: apply_ex (two-pass) +{grew} bytes")
    assert grew >= n[0] * n[1] * n[2] * 4
    used = reset_high()
    for _ in range(2):
        _lib.apply_noalloc(r, c, inp, out, path="bf16x3")
    torch.cuda.synchronize()
    mms.check_device()
    grew = attr(USED_HIGH) - used
    print(f"default pool high-water mark: no-alloc +{grew} bytes")
    assert grew == 0
