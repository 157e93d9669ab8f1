"""The C-ABI library on a machine without a GPU: it builds, loads, exports
every symbol include/mms.h declares, and rejects bad arguments before it
touches the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2507_11067_gb300 as mms
from paper_2507_11067_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    mms.build()
    return mms.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mms.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mms_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_version_and_variants(lib):
    assert "sm_103a" in mms.version()
    assert mms.num_variants("star", 4, "cuda_core") >= 4
    assert mms.num_variants("box", 2, "cuda_core") >= 4
    assert mms.num_variants("star", 5, "cuda_core") == 0
    assert mms.num_variants("box", 1, "naive") == 1


def _desc(**kw):
    c = np.ones(729, np.float32)
    d = _lib.StencilDesc(kw.get("shape", 1), kw.get("radius", 2), c.ctypes.data, kw.get("nx", 8),
                         kw.get("ny", 8), kw.get("nz", 8), kw.get("ipy", 0), kw.get("ipz", 0),
                         kw.get("opy", 0), kw.get("opz", 0), kw.get("path", 0), kw.get("variant", -1))
    return d, c


@pytest.mark.parametrize("kw,status", [
    (dict(radius=0), 1), (dict(radius=5), 1), (dict(shape=9), 1), (dict(shape=-1), 1), (dict(nx=-1), 1),
    (dict(path=9), 1), (dict(ipy=3), 1), (dict(opy=2), 1), (dict(variant=-2), 1),
    # pitches whose products would leave 64 bits, or negative ones
    (dict(ipy=1 << 62), 1), (dict(ipz=1 << 62), 1), (dict(opy=1 << 61), 1), (dict(opz=-16), 1),
    (dict(ipy=-12), 1), (dict(nx=(1 << 30) - 1, ny=(1 << 30) - 1, nz=(1 << 30) - 1), 1),
])
def test_argument_validation(lib, kw, status):
    d, c = _desc(**kw)
    buf_in = ctypes.create_string_buffer(64)
    buf_out = ctypes.create_string_buffer(64)
    st = lib.mms_stencil_apply_ex(ctypes.byref(d), buf_in, buf_out, None)
    assert st == status
    assert lib.mms_last_error()


def test_null_grid_and_overlap_rejected(lib):
    d, c = _desc()
    assert lib.mms_stencil_apply_ex(ctypes.byref(d), None, None, None) == 1
    buf = ctypes.create_string_buffer(1 << 16)
    assert lib.mms_stencil_apply_ex(ctypes.byref(d), buf, buf, None) == 1
    assert b"overlap" in lib.mms_last_error()


def test_empty_interior_is_a_no_op(lib):
    d, c = _desc(nx=0)
    assert lib.mms_stencil_apply_ex(ctypes.byref(d), None, None, None) == 0


def test_wave_validation(lib):
    d, src = mms.wave_desc(8, 8, 8, 4, 0)
    c = np.zeros(27, np.float32)
    assert lib.mms_wave_step(ctypes.byref(d), c.ctypes.data, None, None, None, None, None, None) == 1
    d, src = mms.wave_desc(8, 8, 8, 4, 1, src=[(9, 0, 0)])
    assert lib.mms_wave_step(ctypes.byref(d), c.ctypes.data, None, None, None, None, None, None) == 1
    assert b"source" in lib.mms_last_error()
    d, src = mms.wave_desc(8, 8, 8, 4, 1, pitch_y=17)
    assert lib.mms_wave_step(ctypes.byref(d), c.ctypes.data, None, None, None, None, None, None) == 3


def test_set_variant_range(lib):
    assert lib.mms_set_variant(1, 2, 1, 99) == 1
    assert lib.mms_set_variant(1, 2, 1, 1) == 0
    assert mms.default_variant("box", 2, "cuda_core") == 1
    assert lib.mms_set_variant(1, 2, 1, -1) == 0
    assert mms.default_variant("box", 2, "cuda_core") == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib._build, "LIB", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load()


def test_sum_f64_validation(lib):
    a = np.zeros(64, np.float64)
    out = np.zeros(16, np.float64)
    P = ctypes.c_void_p
    assert lib.mms_sum_f64(a.ctypes.data_as(P), 0, 16, 16, out.ctypes.data_as(P), None) == 1
    assert lib.mms_sum_f64(a.ctypes.data_as(P), 2, 8, 16, out.ctypes.data_as(P), None) == 1
    assert lib.mms_sum_f64(a.ctypes.data_as(P), 2, 16, -1, out.ctypes.data_as(P), None) == 1
    assert lib.mms_sum_f64(a.ctypes.data_as(P), 2, 16, 0, out.ctypes.data_as(P), None) == 0
    # out may be the first slice, not another one
    second = ctypes.c_void_p(a.ctypes.data + 16 * 8)
    assert lib.mms_sum_f64(a.ctypes.data_as(P), 2, 16, 16, second, None) == 1
    assert b"slice 1" in lib.mms_last_error()


def _wave_desc(**kw):
    src = np.array([3, 3, 3], np.int32)
    d, keep = _lib.wave_desc(kw.get("n", 16), kw.get("n", 16), kw.get("n", 16), 4, 1,
                             rec_z=2, src=src, grad_shot_stride=kw.get("gss", 0))
    return d, (keep, src)


def test_wave_gradient_stride_and_step_to_validation(lib):
    c = np.ones(27, np.float32)
    P = ctypes.c_void_p
    buf = [np.zeros(24 ** 3 + 64, np.float32) for _ in range(3)]
    ptr = [b.ctypes.data_as(P) for b in buf]
    d, keep = _wave_desc(gss=100)   # below 16^3
    st = lib.mms_wave_adjoint(ctypes.byref(d), c.ctypes.data_as(P), ptr[0], ptr[1], ptr[2], None, None,
                              None, None)
    assert st == 1 and b"gradient shot stride" in lib.mms_last_error()
    d, keep = _wave_desc()
    # p_next overlapping p_cur, or overlapping p_prev without being it
    st = lib.mms_wave_step_to(ctypes.byref(d), c.ctypes.data_as(P), ptr[0], ptr[1], ptr[2], ptr[1],
                              ptr[0], None, None)
    assert st == 1 and b"p_cur and p_next overlap" in lib.mms_last_error()
    shifted = ctypes.c_void_p(buf[2].ctypes.data + 64)
    st = lib.mms_wave_step_to(ctypes.byref(d), c.ctypes.data_as(P), ptr[0], ptr[1], ptr[2], shifted,
                              ptr[0], None, None)
    assert st == 1 and b"p_prev and p_next overlap" in lib.mms_last_error()


def test_selftest_limit_validation(lib):
    assert lib.mms_selftest_timeout(0, None) == 1
    assert lib.mms_selftest_timeout(2000001, None) == 1


def test_host_sweep_validation(lib):
    d, c = _desc(radius=2)
    a = np.zeros(16, np.float32)
    P = ctypes.c_void_p
    assert lib.mms_stencil_apply_host(ctypes.byref(d), None, a.ctypes.data_as(P), None) == 1
    d, c = _desc(ipy=11)      # below the padded extent
    assert lib.mms_stencil_apply_host(ctypes.byref(d), a.ctypes.data_as(P), a.ctypes.data_as(P), None) == 1
    d, c = _desc(ipy=13)      # not a multiple of 4 floats
    assert lib.mms_stencil_apply_host(ctypes.byref(d), a.ctypes.data_as(P), a.ctypes.data_as(P), None) == 3
    d, c = _desc(nx=0)        # empty interior: nothing to do
    assert lib.mms_stencil_apply_host(ctypes.byref(d), None, None, None) == 0


def test_planar_shapes_are_known(lib):
    assert mms.num_variants("star2d", 2, "cuda_core") > 0
    assert mms.num_variants("box2d", 3, "bf16x3") > 0
    assert lib.mms_auto_path(4, 2, 1) == -1
    d, c = _desc(shape=4)
    buf = ctypes.create_string_buffer(64)
    assert lib.mms_stencil_apply_ex(ctypes.byref(d), buf, buf, None) == 1


def test_f64_sweep_validation(lib):
    P = ctypes.c_void_p
    c = np.ones(729, np.float64)
    a = np.zeros(64, np.float64)
    buf = ctypes.create_string_buffer(1024)
    d, _ = _desc(radius=2)
    assert lib.mms_stencil_apply_f64(ctypes.byref(d), None, a.ctypes.data_as(P), a.ctypes.data_as(P), None) == 1
    assert lib.mms_stencil_apply_f64(ctypes.byref(d), c.ctypes.data_as(P), None, None, None) == 1
    d, _ = _desc(radius=5)
    assert lib.mms_stencil_apply_f64(ctypes.byref(d), c.ctypes.data_as(P), buf, buf, None) == 1
    d, _ = _desc(path=3)      # a tensor-core path: FP64 runs on the CUDA cores only
    assert lib.mms_stencil_apply_f64(ctypes.byref(d), c.ctypes.data_as(P), buf, buf, None) == 2
    d, _ = _desc()
    assert lib.mms_stencil_apply_f64(ctypes.byref(d), c.ctypes.data_as(P), buf, buf, None) == 1   # overlap
    odd = ctypes.c_void_p(ctypes.addressof(buf) + 4)
    assert lib.mms_stencil_apply_f64(ctypes.byref(d), c.ctypes.data_as(P), odd, buf, None) == 3
    d, _ = _desc(nz=0)
    assert lib.mms_stencil_apply_f64(ctypes.byref(d), c.ctypes.data_as(P), None, None, None) == 0


def test_anisotropic_and_lap_outputs_may_not_alias_their_inputs(lib):
    # validation happens before anything is enqueued: host buffers suffice
    P = ctypes.c_void_p
    nx, ny, nz, r = 10, 8, 8, 1          # padded rows of 12 floats: 16-byte pitches
    d, _src = _lib.wave_desc(nx, ny, nz, r, 1)
    fb = (nz + 2 * r) * (ny + 2 * r) * (nx + 2 * r)
    bufs = [np.zeros(fb + 16, np.float32) for _ in range(8)]
    a = [ctypes.c_void_p((b.ctypes.data + 15) & ~15) for b in bufs]
    c = np.ones(9, np.float32).ctypes.data_as(P)
    amp = np.zeros(1, np.float32).ctypes.data_as(P)
    # sh_next over mv
    assert lib.mms_vti_step(ctypes.byref(d), c, a[0], a[1], a[2], a[3], a[4], a[5], a[0], a[6], amp, None, None) == 1
    assert b"medium" in lib.mms_last_error()
    # vti model: mv over vp
    assert lib.mms_vti_model(ctypes.byref(d), a[0], a[1], a[2], a[0], a[3], ctypes.c_float(1e-3),
                             ctypes.c_float(10.0), None) == 1
    # step_lap: lap_out over m
    assert lib.mms_wave_step_lap(ctypes.byref(d), c, a[0], a[1], a[2], a[3], a[0], amp, None, None) == 1
    assert b"overlaps m" in lib.mms_last_error()


def test_wave_outputs_may_not_alias_their_inputs(lib):
    # validation happens before anything is enqueued: host buffers suffice
    P = ctypes.c_void_p
    nx, ny, nz, r = 10, 8, 8, 1
    d, _src = _lib.wave_desc(nx, ny, nz, r, 1, rec_z=0)
    fb = (nz + 2 * r) * (ny + 2 * r) * (nx + 2 * r)
    bufs = [np.zeros(fb + 16, np.float32) for _ in range(6)]
    a = [ctypes.c_void_p((b.ctypes.data + 15) & ~15) for b in bufs]
    c = np.ones(9, np.float32).ctypes.data_as(P)
    amp = np.zeros(4, np.float32).ctypes.data_as(P)

    def refused(status, words):
        assert status == 1
        assert words in lib.mms_last_error(), lib.mms_last_error()

    m, p, q, x, y, z = a
    refused(lib.mms_wave_step(ctypes.byref(d), c, m, p, m, amp, None, None), b"overlaps m")
    refused(lib.mms_wave_step(ctypes.byref(d), c, m, p, q, amp, p, None), b"rec overlaps")
    refused(lib.mms_wave_step_to(ctypes.byref(d), c, m, p, q, m, amp, None, None), b"overlaps m")
    refused(lib.mms_wave_forward(ctypes.byref(d), c, m, amp, 2, m, q, None, None, 1, 0, None), b"overlaps m")
    refused(lib.mms_wave_forward(ctypes.byref(d), c, m, amp, 2, p, q, None, p, 1, 0, None), b"ckpt overlaps")
    refused(lib.mms_wave_forward(ctypes.byref(d), c, m, amp, 2, p, q, m, None, 1, 0, None), b"rec_all overlaps")
    refused(lib.mms_wave_adjoint(ctypes.byref(d), c, m, p, m, None, None, None, None), b"lam_prev overlaps m")
    refused(lib.mms_wave_adjoint(ctypes.byref(d), c, m, p, q, None, x, p, None), b"grad_m overlaps")
    refused(lib.mms_wave_adjoint(ctypes.byref(d), c, m, p, q, q, None, None, None), b"resid overlaps")
    refused(lib.mms_wave_adjoint_scaled(ctypes.byref(d), c, m, p, m, None, None, None, None), b"mu_prev overlaps m")
    refused(lib.mms_wave_adjoint_scaled(ctypes.byref(d), c, m, p, p, None, None, None, None), b"overlap")
    refused(lib.mms_wave_adjoint_scaled(ctypes.byref(d), c, m, p, q, None, x, p, None), b"grad_m overlaps")
    refused(lib.mms_wave_adjoint_scaled(ctypes.byref(d), c, m, p, q, q, None, None, None), b"resid overlaps")
    refused(lib.mms_wave_adjoint_scaled(ctypes.byref(d), c, m, p, q, None, x, None, None), b"without grad_m")
    refused(lib.mms_wave_adjoint_scaled(ctypes.byref(d), c, m, p, q, None, q, P(x.value + 8 * 0), None),
            b"overlap")
    refused(lib.mms_grad_divide_m(ctypes.byref(d), m, P(m.value), None), b"grad_m overlaps m")
    refused(lib.mms_grad_divide_m(ctypes.byref(d), None, x, None), b"null pointer")
    refused(lib.mms_model_from_velocity(ctypes.byref(d), m, m, ctypes.c_float(1e-3), ctypes.c_float(10.0), None),
            b"overlaps v")
    n = nx * ny * nz
    g = np.zeros(n + 8, np.float64)
    gp = g.ctypes.data
    refused(lib.mms_grad_to_velocity(P(gp), x, P(gp + 8), n, ctypes.c_float(1e-3), ctypes.c_float(10.0), None),
            b"grad_v overlaps grad_m")
    refused(lib.mms_grad_to_velocity(P(gp), x, x, n, ctypes.c_float(1e-3), ctypes.c_float(10.0), None),
            b"grad_v overlaps v")
    refused(lib.mms_dot_f64(x, y, n, x, None), b"result overlaps")


def test_tti_work_and_outputs_may_not_alias(lib):
    P = ctypes.c_void_p
    nx, ny, nz, r = 10, 8, 8, 1
    d, _src = _lib.wave_desc(nx, ny, nz, r, 1)
    n = nx * ny * nz
    size = max((nz + 2 * r) * (ny + 2 * r) * (nx + 2 * r), 8 * n)
    bufs = [np.zeros(size + 16, np.float32) for _ in range(8)]
    med, pc, qc, pp, qp, pn, qn, work = [ctypes.c_void_p((b.ctypes.data + 15) & ~15) for b in bufs]
    w = np.ones(3, np.float32).ctypes.data_as(P)
    amp = np.zeros(1, np.float32).ctypes.data_as(P)
    assert lib.mms_tti_step(ctypes.byref(d), w, w, med, pc, qc, pp, qp, pn, qn, pn, amp, None, None) == 1
    assert b"work overlaps" in lib.mms_last_error()
    assert lib.mms_tti_step(ctypes.byref(d), w, w, med, pc, qc, pp, qp, pn, pn, work, amp, None, None) == 1
    assert b"overlap" in lib.mms_last_error()
    assert lib.mms_tti_step(ctypes.byref(d), w, w, med, pc, qc, pp, qp, med, qn, work, amp, None, None) == 1
    assert b"med" in lib.mms_last_error()


def test_spans_beyond_any_device_are_refused(lib):
    # every caller-given pitch and stride is bounded before a product of it
    # is formed (2^46 elements), so no extent check can wrap around
    c = np.zeros(27, np.float32)
    P = ctypes.c_void_p
    buf = ctypes.create_string_buffer(1 << 12)
    for kw in (dict(pitch_y=1 << 62), dict(pitch_z=1 << 62), dict(shot_stride=1 << 62), dict(pitch_y=-16),
               dict(grad_shot_stride=1 << 62)):
        d, _s = mms.wave_desc(8, 8, 8, 4, 2, **kw)
        assert lib.mms_wave_step(ctypes.byref(d), c.ctypes.data, buf, buf, buf, buf, None, None) == 1, kw
        assert b"2^46" in lib.mms_last_error(), kw
    d, _ = _desc(ipy=1 << 62)
    assert lib.mms_stencil_apply_host(ctypes.byref(d), buf, buf, None) == 1
    assert lib.mms_stencil_apply_f64(ctypes.byref(d), c.ctypes.data_as(P), buf, buf, None) == 1
    assert b"2^46" in lib.mms_last_error()
    assert lib.mms_sum_f64(buf, 4, 1 << 62, 8, buf, None) == 1
    assert b"2^46" in lib.mms_last_error()
    assert lib.mms_sum_f64(buf, 1, 0, 1 << 62, buf, None) == 1


def test_every_declaration_is_documented():
    # each entry point of the header sits under a comment block (a group of
    # consecutive declarations may share one)
    lines = open(os.path.join(ROOT, "include", "mms.h")).read().splitlines()
    decl = re.compile(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(mms_[a-z0-9_]+)\s*\(")
    seen = []
    for i, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        j = i - 1
        while j >= 0 and not lines[j].strip():
            j -= 1
        # step back over the declarations of the same group
        while j >= 0 and (lines[j].rstrip().endswith(");") or lines[j].startswith(" ")) \
                and not lines[j].strip().endswith("*/"):
            j -= 1
        assert j >= 0 and lines[j].strip().endswith("*/"), m.group(1)
        seen.append(m.group(1))
    assert sorted(seen) == declared_symbols()
