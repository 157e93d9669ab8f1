"""The Python binding's argument checks, on CPU tensors.

The binding refuses (ArgumentError: an MMSError with MMS_E_ARG that is also
a ValueError) every buffer the library would reach beyond its storage, of
the wrong dtype, not dense where the call reads a dense array, or on the
wrong side of the bus, before it calls the library.  With the device check
replaced, CPU tensors of the sizes the GPU tests use pass both the binding
and the library's own validation and stop at the first CUDA call
(MMS_E_CUDA): the sizes the binding requires are the ones correct callers
pass.  Those calls hand host pointers to the library, so they run only
where there is no GPU.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_11067_gb300 as mms  # noqa: E402
from paper_2507_11067_gb300 import _lib  # noqa: E402

E_ARG, E_CUDA = 1, 4
R = 4


def test_cpu_tensors_are_refused_before_the_library():
    # safe anywhere: the refusal comes before any library call
    inp = mms.padded_empty(20, 12, 9, 2, device="cpu")
    with pytest.raises(_lib.ArgumentError, match="CUDA tensor") as e:
        mms.apply("star", 2, np.ones(15), inp)
    assert e.value.status == E_ARG and isinstance(e.value, ValueError)
    desc, _s = mms.wave_desc(8, 8, 8, 1, 1)
    f = mms.padded_empty(8, 8, 8, 1, device="cpu", nshots=1)
    with pytest.raises(_lib.ArgumentError, match="CUDA tensor"):
        mms.wave_step(desc, np.ones(9), mms.padded_empty(8, 8, 8, 1, device="cpu"), f, f.clone(),
                      torch.zeros(1))


no_gpu = pytest.mark.skipif(torch.cuda.is_available(), reason="hands host pointers to the library")


@pytest.fixture
def host_ok(monkeypatch):
    mms.build()
    mms.load()
    monkeypatch.setattr(_lib, "_device_problem", lambda t: None)


def accepted(fn, *a, **k):
    with pytest.raises(mms.MMSError) as e:
        fn(*a, stream=0, **k)
    assert e.value.status == E_CUDA, str(e.value)


def refused(fn, *a, match=None, **k):
    with pytest.raises(_lib.ArgumentError, match=match):
        fn(*a, stream=0, **k)


@no_gpu
def test_sweep_arguments(host_ok):
    r, (nx, ny, nz) = 2, (20, 12, 9)
    inp = mms.padded_empty(nx, ny, nz, r, device="cpu")
    c = np.ones(15, np.float32)
    accepted(mms.apply, "star", r, c, inp)
    accepted(mms.apply, "box", r, np.ones(125), inp, path="bf16x3")
    refused(mms.apply, "star", r, c[:-1], inp, match="15 weights")
    refused(mms.apply, "star", r, c, inp, torch.empty((nz, ny, nx - 1)), match="shape")
    refused(mms.apply, "star", r, c, inp, torch.empty((nz, ny, nx), dtype=torch.float64), match="float32")
    refused(mms.apply, "star", r, c, inp.double(), match="float32")
    accepted(mms.apply_f64, "star", r, c, mms.padded_empty(nx, ny, nz, r, device="cpu", dtype=torch.float64))
    refused(mms.apply_f64, "star", r, c, inp, match="float64")
    accepted(_lib.apply_noalloc, r, c, inp, path="bf16x3")
    hin = mms.padded_empty(nx, ny, nz, r, device="cpu")
    accepted(mms.apply_host, "star", r, c, hin, torch.empty((nz, ny, nx)))
    refused(mms.apply_host, "star", r, c, hin, torch.empty((nz - 1, ny, nx)), match="shape")
    dense = torch.zeros((nz + 2 * r, ny + 2 * r, nx + 2 * r))
    accepted(mms.apply_dense, "star", r, c, dense, torch.empty((nz, ny, nx)))
    refused(mms.apply_dense, "star", r, c, inp, torch.empty((nz, ny, nx)), match="contiguous")


class Wave:
    """The geometry of the GPU wave tests, in host memory."""

    def __init__(self, nx=45, ny=38, nz=41, ns=3, rec_z=5, gss=0):
        self.nx, self.ny, self.nz, self.ns = nx, ny, nz, ns
        self.m = mms.padded_empty(nx, ny, nz, R, device="cpu")
        self.f = [mms.padded_empty(nx, ny, nz, R, device="cpu", nshots=ns) for _ in range(6)]
        py, pz, ss = mms.field_geometry(self.f[0])
        src = [(1 + k, 2, 3) for k in range(ns)]
        self.desc, self._src = mms.wave_desc(nx, ny, nz, R, ns, py, pz, ss, 6, 0.01, rec_z, src,
                                             grad_shot_stride=gss)
        self.cf = np.ones(27, np.float32)
        self.amp = torch.zeros(ns)
        self.rec = torch.zeros((ns, ny, nx))
        self.n = nx * ny * nz


@no_gpu
def test_wave_arguments(host_ok):
    w = Wave()
    d, cf, m, (a, b, c, e, f, g) = w.desc, w.cf, w.m, w.f
    accepted(mms.wave_step, d, cf, m, a, b, w.amp, w.rec)
    refused(mms.wave_step, d, cf[:9], m, a, b, w.amp, w.rec, match="27 weights")
    refused(mms.wave_step, d, cf, m, a[-1], b, w.amp, w.rec, match="p_cur holds")   # room for one shot
    refused(mms.wave_step, d, cf, m, a, b, w.amp[:1].clone(), w.rec, match="src_amp")
    refused(mms.wave_step, d, cf, m, a, b, w.amp, w.rec[:2].clone(), match="rec holds")
    refused(mms.wave_step, d, cf, m[:, :, :8].contiguous(), a, b, w.amp, match="m holds")
    accepted(mms.wave_step_to, d, cf, m, a, b, c, w.amp)
    accepted(mms.wave_step_lap, d, cf, m, a, b, c, e, w.amp, w.rec)
    refused(mms.wave_step_lap, d, cf, m, a, b, c, e[0].clone(), w.amp, match="lap_out")
    grad = torch.zeros((w.nz, w.ny, w.nx), dtype=torch.float64)
    accepted(mms.wave_adjoint, d, cf, m, a, b, w.rec, c, grad)
    accepted(mms.wave_adjoint_lap, d, cf, m, a, b, w.rec, c, grad)
    refused(mms.wave_adjoint, d, cf, m, a, b, w.rec, c, grad.float(), match="float64")
    refused(mms.wave_adjoint, d, cf, m, a, b, w.rec, c, grad[1:].clone(), match="grad_m holds")
    # per-shot slices: ns of them
    ws = Wave(gss=w.n)
    slices = torch.zeros((w.ns, w.nz, w.ny, w.nx), dtype=torch.float64)
    accepted(mms.wave_adjoint, ws.desc, cf, m, a, b, w.rec, c, slices)
    refused(mms.wave_adjoint, ws.desc, cf, m, a, b, w.rec, c, slices[:2].clone(), match="grad_m holds")
    # the forward sequence: amps and records for every step, checkpoint slots
    nsteps, every = 25, 10
    amps = torch.zeros((nsteps, w.ns))
    rec_all = torch.zeros((nsteps, w.ns, w.ny, w.nx))
    whole = a.untyped_storage().nbytes() // 4
    ckpt = torch.zeros((3, 2, whole))
    for graph in (False, True):
        accepted(mms.wave_forward, d, cf, m, amps, nsteps, a, b, rec_all, ckpt, every, graph=graph)
    refused(mms.wave_forward, d, cf, m, amps, nsteps, a, b, rec_all, ckpt[:2].clone(), every, match="ckpt holds")
    refused(mms.wave_forward, d, cf, m, amps[:-1].clone(), nsteps, a, b, rec_all, ckpt, every, match="amps holds")
    refused(mms.wave_forward, d, cf, m, amps, nsteps, a, b, rec_all[1:].clone(), match="rec_all holds")
    # the medium and the chain rule read dense interiors
    v = torch.ones((w.nz, w.ny, w.nx))
    accepted(mms.model_from_velocity, d, v, m, 1e-3, 10.0)
    refused(mms.model_from_velocity, d, v.transpose(0, 2), m, 1e-3, 10.0, match="contiguous")
    accepted(mms.grad_to_velocity, grad, v, torch.empty_like(grad), 1e-3, 10.0)
    refused(mms.grad_to_velocity, grad, v, torch.empty_like(v), 1e-3, 10.0, match="float64")
    accepted(mms.sum_f64, slices, slices[0])
    refused(mms.sum_f64, slices, torch.zeros(10, dtype=torch.float64), match="out holds")
    x = torch.zeros(100)
    accepted(mms.dot_f64, x, torch.ones(100), torch.zeros(1, dtype=torch.float64))
    refused(mms.dot_f64, x, torch.ones(99), torch.zeros(1, dtype=torch.float64))
    refused(mms.dot_f64, x, torch.ones(100), torch.zeros(1), match="float64")


@no_gpu
def test_anisotropic_arguments(host_ok):
    w = Wave(ns=2)
    d, cf, (a, b, c, e, f, g) = w.desc, w.cf, w.f
    mv, rho = mms.padded_empty(w.nx, w.ny, w.nz, R, device="cpu"), mms.padded_empty(w.nx, w.ny, w.nz, R, device="cpu")
    dense = [torch.ones((w.nz, w.ny, w.nx)) for _ in range(7)]
    accepted(mms.vti_model, d, *dense[:3], mv, rho, 1e-3, 10.0)
    accepted(mms.vti_step, d, cf, mv, rho, a, b, c, e, f, g, w.amp, w.rec)
    accepted(mms.vti_step, d, cf, mv, rho, a, b, c, e, c, e, w.amp)            # in place
    refused(mms.vti_step, d, cf, mv, rho, a, b, c, e, f, g[0].clone(), w.amp, match="sv_next holds")
    med = torch.empty((8, w.nz, w.ny, w.nx))
    work = torch.empty((4, w.ns, w.nz, w.ny, w.nx))
    accepted(mms.tti_model, d, *dense, med, 1e-3, 10.0)
    refused(mms.tti_model, d, *dense, med[:7].clone(), 1e-3, 10.0, match="med holds")
    w2, w1 = np.ones(9), np.ones(9)
    accepted(mms.tti_step, d, w2, w1, med, a, b, c, e, f, g, work, w.amp, w.rec)
    refused(mms.tti_step, d, w2, w1, med, a, b, c, e, f, g, work[:3].clone(), w.amp, match="work holds")
    refused(mms.tti_step, d, w2[:-1], w1, med, a, b, c, e, f, g, work, w.amp, match="9 weights")


@no_gpu
def test_descriptors_the_library_refuses_are_left_to_it(host_ok):
    # 65 shots, or an empty interior: no size rules from the binding; the
    # library itself refuses the descriptor (MMS_E_ARG, not ArgumentError)
    w = Wave(ns=2)
    for bad in (mms.wave_desc(w.nx, w.ny, w.nz, R, 65, *mms.field_geometry(w.f[0]))[0],
                mms.wave_desc(0, w.ny, w.nz, R, 2, *mms.field_geometry(w.f[0]))[0]):
        with pytest.raises(mms.MMSError) as e:
            mms.vti_step(bad, w.cf, w.m, w.m, *w.f, w.amp, stream=0)
        assert e.value.status == E_ARG and not isinstance(e.value, _lib.ArgumentError)
