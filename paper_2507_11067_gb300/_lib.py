"""ctypes binding of libmms.so (include/mms.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  torch tensors provide device memory and the current stream.  If
the shared library has not been built, loading fails with an explicit error;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

STAR, BOX, STAR2D, BOX2D = 0, 1, 2, 3
SHAPES = {"star": STAR, "box": BOX, "star2d": STAR2D, "box2d": BOX2D,
          STAR: STAR, BOX: BOX, STAR2D: STAR2D, BOX2D: BOX2D}
PLANAR = (STAR2D, BOX2D)


def n_coeffs(shape, r):
    """Stored weights of a shape: 3(2r+1) star, (2r+1)^3 box, 2(2r+1) star2d, (2r+1)^2 box2d."""
    w = 2 * r + 1
    return {STAR: 3 * w, BOX: w ** 3, STAR2D: 2 * w, BOX2D: w * w}[SHAPES[shape]]


def interior(shape, r, padded_shape):
    """(nx, ny, nz) of a padded (Z, Y, X) grid: the planar shapes have no z
    halo (nz independent planes)."""
    Z, Y, X = padded_shape
    return X - 2 * r, Y - 2 * r, Z - (0 if SHAPES[shape] in PLANAR else 2 * r)
PATHS = {"auto": 0, "cuda_core": 1, "tf32": 2, "3xtf32": 3, "bf16x3": 4, "naive": 5}
PATH_NAMES = {v: k for k, v in PATHS.items()}
STATUS = {0: "MMS_OK", 1: "MMS_E_ARG", 2: "MMS_E_UNSUPPORTED", 3: "MMS_E_ALIGN", 4: "MMS_E_CUDA",
          5: "MMS_E_TIMEOUT", 6: "MMS_E_DEVICE", 7: "MMS_E_NOMEM"}
WAVE_GRAPH = 1
NOALLOC_MAX_POINTS = 8388608  # MMS_NOALLOC_MAX_POINTS of include/mms.h

# Every symbol include/mms.h declares (checked by the CPU test suite).
EXPORTS = ["mms_stencil_apply", "mms_stencil_apply_ex", "mms_auto_path", "mms_num_variants",
           "mms_default_variant",
           "mms_set_variant", "mms_wave_step", "mms_wave_forward", "mms_wave_adjoint",
           "mms_model_from_velocity", "mms_grad_to_velocity", "mms_dot_f64", "mms_last_error",
           "mms_check_device", "mms_version", "mms_stencil_apply_noalloc", "mms_wave_step_to",
           "mms_sum_f64", "mms_selftest_timeout", "mms_stencil_apply_host", "mms_vti_model", "mms_vti_step",
           "mms_aniso_num_variants", "mms_aniso_set_variant", "mms_tti_model", "mms_tti_step", "mms_stencil_apply_f64", "mms_wave_step_lap",
           "mms_wave_adjoint_lap", "mms_wave_adjoint_scaled", "mms_grad_divide_m", "mms_tc_pipeline_config"]


MAX_SHOTS = 64  # largest mms_wave_desc.nshots the library takes


class MMSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ArgumentError(MMSError, ValueError):
    """An argument the binding refuses before calling the library (status
    MMS_E_ARG): a buffer of the wrong type, place or size."""

    def __init__(self, msg: str):
        super().__init__(1, msg)


def _extent(t) -> int:
    """Bytes from the view's first element to the end of its storage."""
    st = t.untyped_storage()
    return st.data_ptr() + st.nbytes() - t.data_ptr()


def _device_problem(t):
    """Why t cannot be handed to a kernel on the current CUDA device, or None."""
    import torch
    if not t.is_cuda:
        return "must be a CUDA tensor"
    cur = torch.cuda.current_device()
    if t.device.index != cur:
        return f"is on {t.device}, the kernels run on cuda:{cur}"
    return None


def _need(t, name, dtype=None, nbytes=0, required=True, dense=False, host=False):
    """Refuse a buffer the library cannot use: of another dtype, not dense
    where the call reads it as a dense array, too short for the nbytes the
    call touches from its first element, or on the wrong side (a CUDA tensor
    of the current device; with host=True, a CPU tensor)."""
    import torch
    if t is None:
        if required:
            raise ArgumentError(f"{name} is required")
        return
    if not isinstance(t, torch.Tensor):
        raise ArgumentError(f"{name} must be a torch tensor, not {type(t).__name__}")
    dtype = dtype or torch.float32
    if t.dtype != dtype:
        raise ArgumentError(f"{name} must be {dtype}, not {t.dtype}")
    if dense and not t.is_contiguous():
        raise ArgumentError(f"{name} must be contiguous")
    if nbytes > 0 and _extent(t) < nbytes:
        raise ArgumentError(f"{name} holds {_extent(t)} bytes from its first element; the call touches {nbytes}")
    if host:
        if t.is_cuda:
            raise ArgumentError(f"{name} must be a CPU tensor")
    else:
        why = _device_problem(t)
        if why:
            raise ArgumentError(f"{name} {why}")


def _need_shape(t, name, shape):
    if tuple(t.shape) != tuple(shape):
        raise ArgumentError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


class StencilDesc(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("radius", ctypes.c_int32),
                ("coeffs", ctypes.c_void_p), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("nz", ctypes.c_int64), ("in_pitch_y", ctypes.c_int64),
                ("in_pitch_z", ctypes.c_int64), ("out_pitch_y", ctypes.c_int64),
                ("out_pitch_z", ctypes.c_int64), ("path", ctypes.c_int32),
                ("variant", ctypes.c_int32)]


class WaveDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("radius", ctypes.c_int32), ("nshots", ctypes.c_int32),
                ("pitch_y", ctypes.c_int64), ("pitch_z", ctypes.c_int64),
                ("shot_stride", ctypes.c_int64), ("sponge_width", ctypes.c_int32),
                ("sponge_a", ctypes.c_float), ("rec_z", ctypes.c_int32),
                ("src_xyz", ctypes.c_void_p), ("grad_shot_stride", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libmms.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run "
                               "paper_2507_11067_gb300.build.build() (or __graft_entry__.build()) first")
        lib = ctypes.CDLL(path)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        sig = {
            "mms_stencil_apply": [i32, i32, P, P, P, i64, i64, i64, P],
            "mms_stencil_apply_ex": [ctypes.POINTER(StencilDesc), P, P, P],
            "mms_stencil_apply_noalloc": [ctypes.POINTER(StencilDesc), P, P, P],
            "mms_stencil_apply_host": [ctypes.POINTER(StencilDesc), P, P, P],
            "mms_stencil_apply_f64": [ctypes.POINTER(StencilDesc), P, P, P, P],
            "mms_num_variants": [i32, i32, i32],
            "mms_tc_pipeline_config": [i32, i32, i32, P, i32],
            "mms_auto_path": [i32, i32, i32],
            "mms_default_variant": [i32, i32, i32, i64, i64, i64],
            "mms_set_variant": [i32, i32, i32, i32],
            "mms_wave_step": [ctypes.POINTER(WaveDesc), P, P, P, P, P, P, P],
            "mms_wave_step_to": [ctypes.POINTER(WaveDesc), P, P, P, P, P, P, P, P],
            "mms_sum_f64": [P, i32, i64, i64, P, P],
            "mms_selftest_timeout": [ctypes.c_uint32, P],
            "mms_wave_forward": [ctypes.POINTER(WaveDesc), P, P, P, i32, P, P, P, P, i32,
                                 ctypes.c_uint32, P],
            "mms_wave_adjoint": [ctypes.POINTER(WaveDesc), P, P, P, P, P, P, P, P],
            "mms_wave_adjoint_lap": [ctypes.POINTER(WaveDesc), P, P, P, P, P, P, P, P],
            "mms_wave_adjoint_scaled": [ctypes.POINTER(WaveDesc), P, P, P, P, P, P, P, P],
            "mms_grad_divide_m": [ctypes.POINTER(WaveDesc), P, P, P],
            "mms_wave_step_lap": [ctypes.POINTER(WaveDesc), P, P, P, P, P, P, P, P, P],
            "mms_model_from_velocity": [ctypes.POINTER(WaveDesc), P, P, ctypes.c_float,
                                        ctypes.c_float, P],
            "mms_grad_to_velocity": [P, P, P, i64, ctypes.c_float, ctypes.c_float, P],
            "mms_dot_f64": [P, P, i64, P, P],
            "mms_vti_model": [ctypes.POINTER(WaveDesc), P, P, P, P, P, ctypes.c_float, ctypes.c_float, P],
            "mms_vti_step": [ctypes.POINTER(WaveDesc), P, P, P, P, P, P, P, P, P, P, P, P],
            "mms_tti_model": [ctypes.POINTER(WaveDesc), P, P, P, P, P, P, P, P, ctypes.c_float, ctypes.c_float,
                              P],
            "mms_tti_step": [ctypes.POINTER(WaveDesc), P, P, P, P, P, P, P, P, P, P, P, P, P],
            "mms_aniso_num_variants": [i32],
            "mms_aniso_set_variant": [i32, i32],
            "mms_last_error": [],
            "mms_check_device": [P],
            "mms_version": [],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int32
        lib.mms_last_error.restype = ctypes.c_char_p
        lib.mms_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def check(status: int):
    if status != 0:
        raise MMSError(status, load().mms_last_error().decode())


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(None)
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream))


def _f64():
    import torch
    return torch.float64


def _host_coeffs(coeffs, count=None, dtype=np.float32) -> np.ndarray:
    """The weights as a contiguous host array; with count, refused unless it
    holds exactly that many (the library reads count values)."""
    c = coeffs
    if hasattr(c, "detach"):
        c = c.detach().cpu().numpy()
    c = np.ascontiguousarray(np.asarray(c, dtype=dtype).reshape(-1))
    if count is not None and c.size != count:
        raise ArgumentError(f"{count} weights expected, got {c.size}")
    return c


# ------------------------------------------------------------ allocation

def padded_empty(nx, ny, nz, r, device="cuda", align=32, nshots=None, dtype=None, zero=True):
    """A padded grid view (nz+2r, ny+2r, nx+2r) over storage whose row pitch
    is rounded up to `align` elements (the TMA paths need 16-byte pitches);
    with nshots, a (nshots, ...) stack.  The halo (and pad) start at zero."""
    import torch
    dtype = dtype or torch.float32
    X, Y, Z = nx + 2 * r, ny + 2 * r, nz + 2 * r
    py = -(-X // align) * align
    shape = (Z, Y, py) if nshots is None else (nshots, Z, Y, py)
    base = (torch.zeros if zero else torch.empty)(shape, device=device, dtype=dtype)
    return base[..., :X]


def pitches(t):
    """(pitch_y, pitch_z) in elements of a 3D (z, y, x) view with unit x stride."""
    if t.dim() != 3 or t.stride(2) != 1:
        raise ValueError("expected a 3D (z, y, x) tensor with unit x stride")
    return t.stride(1), t.stride(0)


def padded_empty2d(nx, ny, nz, r, device="cuda", align=32, zero=True):
    """nz planes padded by r in x and y only: a (nz, ny+2r, nx+2r) view over
    storage whose row pitch is rounded up to `align` elements."""
    import torch
    X, Y = nx + 2 * r, ny + 2 * r
    py = -(-X // align) * align
    base = (torch.zeros if zero else torch.empty)((nz, Y, py), device=device, dtype=torch.float32)
    return base[..., :X]


def to_padded_device2d(grid: np.ndarray, r: int, device="cuda", align=32):
    """Copy host planes (nz, ny+2r, nx+2r) into a pitched device view."""
    import torch
    Z, Y, X = grid.shape
    t = padded_empty2d(X - 2 * r, Y - 2 * r, Z, r, device=device, align=align, zero=False)
    t.copy_(torch.from_numpy(np.ascontiguousarray(grid, dtype=np.float32)))
    return t


def to_padded_device(grid: np.ndarray, r: int, device="cuda", align=32):
    """Copy a host padded grid (nz+2r, ny+2r, nx+2r) into a pitched device view."""
    import torch
    Z, Y, X = grid.shape
    t = padded_empty(X - 2 * r, Y - 2 * r, Z - 2 * r, r, device=device, align=align, zero=False)
    t.copy_(torch.from_numpy(np.ascontiguousarray(grid, dtype=np.float32)))
    return t


# ---------------------------------------------------------------- sweeps

def apply(shape, r, coeffs, inp, out=None, path="auto", variant=-1, stream=None):
    """One stencil sweep: out(x,y,z) = sum_d c_d in(x+r+dx, ...) (mms_stencil_apply_ex).

    inp: CUDA float32 (nz+2r, ny+2r, nx+2r) view with unit x stride (any
    pitches); out: (nz, ny, nx) view or None (allocated).  Returns out.
    """
    import torch
    _need(inp, "input")
    nx, ny, nz = interior(shape, r, inp.shape)
    if out is None:
        out = torch.empty((nz, ny, nx), device=inp.device, dtype=torch.float32)
    _need(out, "output")
    _need_shape(out, "output", (nz, ny, nx))
    ipy, ipz = pitches(inp)
    opy, opz = pitches(out)
    c = _host_coeffs(coeffs, n_coeffs(shape, r))
    d = StencilDesc(SHAPES[shape], r, c.ctypes.data, nx, ny, nz, ipy, ipz, opy, opz,
                    PATHS[path] if isinstance(path, str) else int(path), int(variant))
    check(load().mms_stencil_apply_ex(ctypes.byref(d), _ptr(inp), _ptr(out), _stream(stream)))
    return out


def apply_f64(shape, r, coeffs, inp, out=None, stream=None):
    """The FP64 sweep (mms_stencil_apply_f64): inp a CUDA float64 padded view
    with unit x stride (any pitches), out an interior view or None."""
    import torch
    _need(inp, "input", torch.float64)
    nx, ny, nz = interior(shape, r, inp.shape)
    if out is None:
        out = torch.empty((nz, ny, nx), device=inp.device, dtype=torch.float64)
    _need(out, "output", torch.float64)
    _need_shape(out, "output", (nz, ny, nx))
    ipy, ipz = pitches(inp)
    opy, opz = pitches(out)
    c = _host_coeffs(coeffs, n_coeffs(shape, r), np.float64)
    d = StencilDesc(SHAPES[shape], r, None, nx, ny, nz, ipy, ipz, opy, opz, PATHS["auto"], -1)
    check(load().mms_stencil_apply_f64(ctypes.byref(d), c.ctypes.data_as(ctypes.c_void_p), _ptr(inp), _ptr(out),
                                       _stream(stream)))
    return out


def apply_noalloc(r, coeffs, inp, out=None, path="bf16x3", variant=-1, stream=None):
    """The star sweep on tensor cores with no device allocation inside the
    call (mms_stencil_apply_noalloc); same arguments as ``apply`` with
    shape "star".  Interiors above NOALLOC_MAX_POINTS points are refused."""
    import torch
    _need(inp, "input")
    nx, ny, nz = interior("star", r, inp.shape)
    if out is None:
        out = torch.empty((nz, ny, nx), device=inp.device, dtype=torch.float32)
    _need(out, "output")
    _need_shape(out, "output", (nz, ny, nx))
    ipy, ipz = pitches(inp)
    opy, opz = pitches(out)
    c = _host_coeffs(coeffs, n_coeffs("star", r))
    d = StencilDesc(SHAPES["star"], r, c.ctypes.data, nx, ny, nz, ipy, ipz, opy, opz,
                    PATHS[path] if isinstance(path, str) else int(path), int(variant))
    check(load().mms_stencil_apply_noalloc(ctypes.byref(d), _ptr(inp), _ptr(out), _stream(stream)))
    return out


def apply_host(shape, r, coeffs, host_in, host_out, path="auto", variant=-1, stream=None):
    """The sweep on grids in host memory (mms_stencil_apply_host): host_in a
    CPU float32 (nz+2r, ny+2r, nx+2r) view with unit x stride (pinned for
    overlapped copies), host_out a CPU (nz, ny, nx) view; the library streams
    z-slabs through the device.  Asynchronous on `stream`."""
    _need(host_in, "host_in", host=True)
    _need(host_out, "host_out", host=True)
    nx, ny, nz = interior(shape, r, host_in.shape)
    _need_shape(host_out, "host_out", (nz, ny, nx))
    ipy, ipz = pitches(host_in)
    opy, opz = pitches(host_out)
    c = _host_coeffs(coeffs, n_coeffs(shape, r))
    d = StencilDesc(SHAPES[shape], r, c.ctypes.data, nx, ny, nz, ipy, ipz, opy, opz,
                    PATHS[path] if isinstance(path, str) else int(path), int(variant))
    check(load().mms_stencil_apply_host(ctypes.byref(d), _ptr(host_in), _ptr(host_out), _stream(stream)))
    return host_out


def apply_dense(shape, r, coeffs, inp, out, stream=None):
    """mms_stencil_apply on dense contiguous tensors (AUTO path)."""
    _need(inp, "input", dense=True)
    nx, ny, nz = interior(shape, r, inp.shape)
    _need(out, "output", dense=True)
    _need_shape(out, "output", (nz, ny, nx))
    c = _host_coeffs(coeffs, n_coeffs(shape, r))
    check(load().mms_stencil_apply(SHAPES[shape], r, c.ctypes.data_as(ctypes.c_void_p), _ptr(inp),
                                   _ptr(out), nx, ny, nz, _stream(stream)))
    return out


def num_variants(shape, r, path) -> int:
    return load().mms_num_variants(SHAPES[shape], r, PATHS[path])


TC_PIPELINE_KEYS = ("mixed", "look", "a_ring", "staging", "accumulators", "reach", "z_halo", "two_ctas",
                    "drainers")


def tc_pipeline_config(shape, r, path):
    """The pipeline constants of the tensor-core sweep of (shape, r, path) in
    this build (mms_tc_pipeline_config), as a dict; None where there is no
    tensor-core sweep.  Needs no GPU."""
    buf = (ctypes.c_int32 * len(TC_PIPELINE_KEYS))()
    n = load().mms_tc_pipeline_config(SHAPES[shape], r, PATHS[path], ctypes.cast(buf, ctypes.c_void_p),
                                      len(TC_PIPELINE_KEYS))
    if n < 0:
        return None
    return dict(zip(TC_PIPELINE_KEYS, list(buf)[:min(n, len(TC_PIPELINE_KEYS))]))


def auto_path(shape, r, tma_aligned=True) -> str:
    """Name of the path MMS_PATH_AUTO takes for (shape, r)."""
    return PATH_NAMES[load().mms_auto_path(SHAPES[shape], r, 1 if tma_aligned else 0)]


def default_variant(shape, r, path, nx=0, ny=0, nz=0) -> int:
    return load().mms_default_variant(SHAPES[shape], r, PATHS[path], nx, ny, nz)


def set_variant(shape, r, path, variant):
    check(load().mms_set_variant(SHAPES[shape], r, PATHS[path], int(variant)))


def check_device(stream=None):
    check(load().mms_check_device(_stream(stream)))


def version() -> str:
    return load().mms_version().decode()


# ------------------------------------------------------------------ wave

def wave_desc(nx, ny, nz, r, nshots, pitch_y=0, pitch_z=0, shot_stride=0, sponge_width=0,
              sponge_a=0.0, rec_z=-1, src=None, grad_shot_stride=0):
    """A WaveDesc plus the host source array it points to (keep both alive)."""
    src_arr = None
    if src is not None:
        src_arr = np.ascontiguousarray(np.asarray(src, dtype=np.int32).reshape(-1))
        if src_arr.size != 3 * nshots:
            raise ValueError("src needs 3 coordinates per shot")
    d = WaveDesc(nx, ny, nz, r, nshots, pitch_y, pitch_z, shot_stride, sponge_width,
                 float(sponge_a), rec_z, None if src_arr is None else src_arr.ctypes.data,
                 int(grad_shot_stride))
    return d, src_arr


class _WaveExtent:
    """Bytes each buffer of a wave call touches, from the geometry of its
    descriptor.  A descriptor the library refuses anyway (sizes, radius or
    shot count out of range) gets no size requirements here: the library
    reports it before it touches any buffer."""

    def __init__(self, desc):
        r, ns = desc.radius, desc.nshots
        self.ok = 1 <= r <= 4 and min(desc.nx, desc.ny, desc.nz) >= 1 and 1 <= ns <= MAX_SHOTS
        X, Y, Z = desc.nx + 2 * r, desc.ny + 2 * r, desc.nz + 2 * r
        py = desc.pitch_y or X
        pz = desc.pitch_z or Y * py
        ss = desc.shot_stride or Z * pz
        one = (Z - 1) * pz + (Y - 1) * py + X          # elements of one padded field the kernels reach
        self.n = desc.nx * desc.ny * desc.nz
        self.shot_stride = ss
        gss = desc.grad_shot_stride
        k = 1 if self.ok else 0
        self.model = k * 4 * one
        self.field = k * 4 * ((ns - 1) * ss + one)
        self.whole_field = k * 4 * ns * ss           # what a checkpoint copy moves
        self.rec = k * 4 * ns * desc.ny * desc.nx
        self.amp = k * 4 * ns
        self.grad = k * 8 * ((ns - 1) * gss + self.n if gss else self.n)
        self.dense = k * 4 * self.n


def _wave_coeffs(desc, coeffs):
    return _host_coeffs(coeffs, 3 * (2 * desc.radius + 1))


def field_geometry(fields):
    """(pitch_y, pitch_z, shot_stride) of a (nshots, Z, Y, X) stacked view."""
    if fields.dim() != 4 or fields.stride(3) != 1:
        raise ValueError("expected a (nshots, z, y, x) view with unit x stride")
    return fields.stride(2), fields.stride(1), fields.stride(0)


def wave_step(desc, coeffs, m, p_cur, p_prev, src_amp, rec=None, stream=None):
    x = _WaveExtent(desc)
    _need(m, "m", nbytes=x.model)
    for t, name in ((p_cur, "p_cur"), (p_prev, "p_prev")):
        _need(t, name, nbytes=x.field)
    _need(src_amp, "src_amp", nbytes=x.amp)
    _need(rec, "rec", nbytes=x.rec, required=False)
    c = _wave_coeffs(desc, coeffs)
    check(load().mms_wave_step(ctypes.byref(desc), c.ctypes.data_as(ctypes.c_void_p), _ptr(m),
                               _ptr(p_cur), _ptr(p_prev), _ptr(src_amp), _ptr(rec),
                               _stream(stream)))


def wave_step_to(desc, coeffs, m, p_cur, p_prev, p_next, src_amp, rec=None, stream=None):
    """mms_wave_step_to: a^{n+1} into p_next, p_prev read only."""
    x = _WaveExtent(desc)
    _need(m, "m", nbytes=x.model)
    for t, name in ((p_cur, "p_cur"), (p_prev, "p_prev"), (p_next, "p_next")):
        _need(t, name, nbytes=x.field)
    _need(src_amp, "src_amp", nbytes=x.amp)
    _need(rec, "rec", nbytes=x.rec, required=False)
    c = _wave_coeffs(desc, coeffs)
    check(load().mms_wave_step_to(ctypes.byref(desc), c.ctypes.data_as(ctypes.c_void_p), _ptr(m),
                                  _ptr(p_cur), _ptr(p_prev), _ptr(p_next), _ptr(src_amp), _ptr(rec),
                                  _stream(stream)))


def wave_forward(desc, coeffs, m, amps, nsteps, p0, p1, rec_all=None, ckpt=None, ckpt_every=0,
                 graph=False, stream=None):
    x = _WaveExtent(desc)
    nsteps, every = int(nsteps), int(ckpt_every)
    steps = max(nsteps, 0)
    _need(m, "m", nbytes=x.model)
    for t, name in ((p0, "p0"), (p1, "p1")):
        _need(t, name, nbytes=x.whole_field if ckpt is not None else x.field)
    _need(amps, "amps", nbytes=steps * x.amp)
    _need(rec_all, "rec_all", nbytes=steps * x.rec, required=False)
    if ckpt is not None and every >= 1:
        _need(ckpt, "ckpt", nbytes=-(-steps // every) * 2 * x.whole_field)
    else:
        _need(ckpt, "ckpt", required=False)
    c = _wave_coeffs(desc, coeffs)
    check(load().mms_wave_forward(ctypes.byref(desc), c.ctypes.data_as(ctypes.c_void_p), _ptr(m),
                                  _ptr(amps), int(nsteps), _ptr(p0), _ptr(p1), _ptr(rec_all),
                                  _ptr(ckpt), int(ckpt_every), WAVE_GRAPH if graph else 0,
                                  _stream(stream)))


def wave_adjoint(desc, coeffs, m, lam_cur, lam_prev, resid=None, a_n=None, grad_m=None,
                 stream=None):
    x = _WaveExtent(desc)
    _need(m, "m", nbytes=x.model)
    for t, name in ((lam_cur, "lam_cur"), (lam_prev, "lam_prev")):
        _need(t, name, nbytes=x.field)
    _need(resid, "resid", nbytes=x.rec, required=False)
    _need(a_n, "a_n", nbytes=x.field, required=False)
    _need(grad_m, "grad_m", _f64(), nbytes=x.grad, required=False)
    c = _wave_coeffs(desc, coeffs)
    check(load().mms_wave_adjoint(ctypes.byref(desc), c.ctypes.data_as(ctypes.c_void_p), _ptr(m),
                                  _ptr(lam_cur), _ptr(lam_prev), _ptr(resid), _ptr(a_n),
                                  _ptr(grad_m), _stream(stream)))


def wave_step_lap(desc, coeffs, m, p_cur, p_prev, p_next, lap_out, src_amp, rec=None, stream=None):
    """mms_wave_step_lap: a^{n+1} into p_next and L a^n into lap_out."""
    x = _WaveExtent(desc)
    _need(m, "m", nbytes=x.model)
    for t, name in ((p_cur, "p_cur"), (p_prev, "p_prev"), (p_next, "p_next"), (lap_out, "lap_out")):
        _need(t, name, nbytes=x.field)
    _need(src_amp, "src_amp", nbytes=x.amp)
    _need(rec, "rec", nbytes=x.rec, required=False)
    c = _wave_coeffs(desc, coeffs)
    check(load().mms_wave_step_lap(ctypes.byref(desc), c.ctypes.data_as(ctypes.c_void_p), _ptr(m), _ptr(p_cur),
                                   _ptr(p_prev), _ptr(p_next), _ptr(lap_out), _ptr(src_amp), _ptr(rec),
                                   _stream(stream)))


def wave_adjoint_lap(desc, coeffs, m, lam_cur, lam_prev, resid=None, lap_a=None, grad_m=None, stream=None):
    """mms_wave_adjoint_lap: the adjoint step with the gradient term from L a^n."""
    x = _WaveExtent(desc)
    _need(m, "m", nbytes=x.model)
    for t, name in ((lam_cur, "lam_cur"), (lam_prev, "lam_prev")):
        _need(t, name, nbytes=x.field)
    _need(resid, "resid", nbytes=x.rec, required=False)
    _need(lap_a, "lap_a", nbytes=x.field, required=False)
    _need(grad_m, "grad_m", _f64(), nbytes=x.grad, required=False)
    c = _wave_coeffs(desc, coeffs)
    check(load().mms_wave_adjoint_lap(ctypes.byref(desc), c.ctypes.data_as(ctypes.c_void_p), _ptr(m),
                                      _ptr(lam_cur), _ptr(lam_prev), _ptr(resid), _ptr(lap_a), _ptr(grad_m),
                                      _stream(stream)))


def wave_adjoint_scaled(desc, coeffs, m, mu_cur, mu_prev, resid=None, lap_a=None, grad_m=None, stream=None):
    """mms_wave_adjoint_scaled: the adjoint step in mu = m G lam (m > 0); its
    gradient sum is m dJ/dm (grad_divide_m turns it into dJ/dm)."""
    x = _WaveExtent(desc)
    _need(m, "m", nbytes=x.model)
    for t, name in ((mu_cur, "mu_cur"), (mu_prev, "mu_prev")):
        _need(t, name, nbytes=x.field)
    _need(resid, "resid", nbytes=x.rec, required=False)
    _need(lap_a, "lap_a", nbytes=x.field, required=False)
    _need(grad_m, "grad_m", _f64(), nbytes=x.grad, required=False)
    c = _wave_coeffs(desc, coeffs)
    check(load().mms_wave_adjoint_scaled(ctypes.byref(desc), c.ctypes.data_as(ctypes.c_void_p), _ptr(m),
                                         _ptr(mu_cur), _ptr(mu_prev), _ptr(resid), _ptr(lap_a), _ptr(grad_m),
                                         _stream(stream)))


def grad_divide_m(desc, m, grad_m, stream=None):
    """mms_grad_divide_m: grad_m /= m at every interior point (FP64)."""
    x = _WaveExtent(desc)
    _need(m, "m", nbytes=x.model)
    _need(grad_m, "grad_m", _f64(), nbytes=x.dense * 2, dense=True)
    check(load().mms_grad_divide_m(ctypes.byref(desc), _ptr(m), _ptr(grad_m), _stream(stream)))


def model_from_velocity(desc, v, m, dt, h, stream=None):
    x = _WaveExtent(desc)
    _need(v, "v", nbytes=x.dense, dense=True)
    _need(m, "m", nbytes=x.model)
    check(load().mms_model_from_velocity(ctypes.byref(desc), _ptr(v), _ptr(m), float(dt),
                                         float(h), _stream(stream)))


def grad_to_velocity(grad_m, v, grad_v, dt, h, stream=None):
    _need(grad_m, "grad_m", _f64(), dense=True)
    n = grad_m.numel()
    _need(v, "v", nbytes=4 * n, dense=True)
    _need(grad_v, "grad_v", _f64(), nbytes=8 * n, dense=True)
    check(load().mms_grad_to_velocity(_ptr(grad_m), _ptr(v), _ptr(grad_v), grad_m.numel(),
                                      float(dt), float(h), _stream(stream)))


def vti_model(desc, vp, eps, delta, mv, rho, dt, h, stream=None):
    """mms_vti_model: the padded VTI medium (mv, rho) from dense vp, eps, delta."""
    x = _WaveExtent(desc)
    for t, name in ((vp, "vp"), (eps, "eps"), (delta, "delta")):
        _need(t, name, nbytes=x.dense, dense=True)
    for t, name in ((mv, "mv"), (rho, "rho")):
        _need(t, name, nbytes=x.model)
    check(load().mms_vti_model(ctypes.byref(desc), _ptr(vp), _ptr(eps), _ptr(delta), _ptr(mv), _ptr(rho),
                               float(dt), float(h), _stream(stream)))


def vti_step(desc, coeffs, mv, rho, sh_cur, sv_cur, sh_prev, sv_prev, sh_next, sv_next, src_amp, rec=None,
             stream=None):
    """mms_vti_step: (sigma_H, sigma_V)^{n+1} into sh_next, sv_next (which may
    be sh_prev, sv_prev)."""
    x = _WaveExtent(desc)
    for t, name in ((mv, "mv"), (rho, "rho")):
        _need(t, name, nbytes=x.model)
    for t, name in ((sh_cur, "sh_cur"), (sv_cur, "sv_cur"), (sh_prev, "sh_prev"), (sv_prev, "sv_prev"),
                    (sh_next, "sh_next"), (sv_next, "sv_next")):
        _need(t, name, nbytes=x.field)
    _need(src_amp, "src_amp", nbytes=x.amp)
    _need(rec, "rec", nbytes=x.rec, required=False)
    c = _wave_coeffs(desc, coeffs)
    check(load().mms_vti_step(ctypes.byref(desc), c.ctypes.data_as(ctypes.c_void_p), _ptr(mv), _ptr(rho),
                              _ptr(sh_cur), _ptr(sv_cur), _ptr(sh_prev), _ptr(sv_prev), _ptr(sh_next),
                              _ptr(sv_next), _ptr(src_amp), _ptr(rec), _stream(stream)))


def tti_model(desc, vp, vs, eps, delta, alpha, theta, phi, med, dt, h, stream=None):
    """mms_tti_model: med (8, nz, ny, nx) = [a, b, c, d, alpha, nx, ny, nz]."""
    x = _WaveExtent(desc)
    for t, name in ((vp, "vp"), (vs, "vs"), (eps, "eps"), (delta, "delta"), (alpha, "alpha"), (theta, "theta"),
                    (phi, "phi")):
        _need(t, name, nbytes=x.dense, dense=True)
    _need(med, "med", nbytes=8 * x.dense, dense=True)
    check(load().mms_tti_model(ctypes.byref(desc), _ptr(vp), _ptr(vs), _ptr(eps), _ptr(delta), _ptr(alpha),
                               _ptr(theta), _ptr(phi), _ptr(med), float(dt), float(h), _stream(stream)))


def tti_step(desc, w2, w1, med, p_cur, q_cur, p_prev, q_prev, p_next, q_next, work, src_amp, rec=None,
             stream=None):
    """mms_tti_step: (p, q)^{n+1} into p_next, q_next (which may be p_prev,
    q_prev); work: 4*nshots*nx*ny*nz floats of scratch."""
    x = _WaveExtent(desc)
    a2, a1 = _host_coeffs(w2, 2 * desc.radius + 1), _host_coeffs(w1, 2 * desc.radius + 1)
    _need(med, "med", nbytes=8 * x.dense, dense=True)
    for t, name in ((p_cur, "p_cur"), (q_cur, "q_cur"), (p_prev, "p_prev"), (q_prev, "q_prev"),
                    (p_next, "p_next"), (q_next, "q_next")):
        _need(t, name, nbytes=x.field)
    _need(work, "work", nbytes=4 * desc.nshots * x.dense if x.ok else 0, dense=True)
    _need(src_amp, "src_amp", nbytes=x.amp)
    _need(rec, "rec", nbytes=x.rec, required=False)
    check(load().mms_tti_step(ctypes.byref(desc), a2.ctypes.data_as(ctypes.c_void_p),
                              a1.ctypes.data_as(ctypes.c_void_p), _ptr(med), _ptr(p_cur), _ptr(q_cur),
                              _ptr(p_prev), _ptr(q_prev), _ptr(p_next), _ptr(q_next), _ptr(work), _ptr(src_amp),
                              _ptr(rec), _stream(stream)))


ANISO_KINDS = {"vti": 0}


def aniso_num_variants(kind="vti"):
    return int(load().mms_aniso_num_variants(ANISO_KINDS[kind]))


def aniso_set_variant(kind, variant):
    check(load().mms_aniso_set_variant(ANISO_KINDS[kind], int(variant)))


def sum_f64(slices, out, stream=None):
    """out = slices.sum(0) in FP64 (mms_sum_f64); slices (k, ...) contiguous,
    out a tensor of the slice shape (may be slices[0])."""
    _need(slices, "slices", _f64())
    k = slices.shape[0]
    n = slices[0].numel()
    if not slices[0].is_contiguous():
        raise ArgumentError("each slice must be contiguous")
    _need(slices, "slices", _f64(), nbytes=8 * ((k - 1) * slices.stride(0) + n))
    _need(out, "out", _f64(), nbytes=8 * n, dense=True)
    check(load().mms_sum_f64(_ptr(slices), int(k), slices.stride(0), n, _ptr(out), _stream(stream)))
    return out


def selftest_timeout(limit_us, stream=None):
    """Queue the failure-path self-test (mms_selftest_timeout): a kernel
    whose bounded wait runs out after limit_us; mms_check_device then
    reports MMS_E_TIMEOUT."""
    check(load().mms_selftest_timeout(int(limit_us), _stream(stream)))


def dot_f64(a, b, result, stream=None):
    _need(a, "a", dense=True)
    _need(b, "b", nbytes=4 * a.numel(), dense=True)
    if b.numel() != a.numel():
        raise ArgumentError(f"a has {a.numel()} values, b {b.numel()}")
    _need(result, "result", _f64(), nbytes=8)
    check(load().mms_dot_f64(_ptr(a), _ptr(b), a.numel(), _ptr(result), _stream(stream)))
