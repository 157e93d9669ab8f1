"""Batched multi-shot acoustic propagation and its adjoint gradient.

The forward model is the damped leapfrog step of mms_wave_step (star
stencil of radius r, Cerjan sponge, one point source per shot, receivers on
one z plane); the paper names reverse time migration with radius-4 stencils
as its application (Sec. 2.1, Sec. 5.6).  ``WaveFunction`` exposes the
records d(v) to torch.autograd: its backward runs the discrete adjoint
(mms_wave_adjoint) over checkpointed segments, recomputing each segment's
states from the checkpoint stored every ``ckpt_every`` steps, and returns
dJ/dv = dJ/dm * 2 v dt^2 / h^2 with dJ/dm accumulated in FP64.  Every step
runs in the library's kernels; torch provides memory and streams.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib


class WavePropagator:
    """Fields, geometry and coefficients of one multi-shot acoustic problem.

    nx, ny, nz: interior size; src: (nshots, 3) interior source points;
    rec_z: receiver plane; h: grid spacing (m); dt: time step (s);
    coeffs: (3, 2r+1) star weights (unscaled; FD8 by default);
    adjoint: the adjoint state the gradient carries: "lam", "mu" (= m G lam,
    mms_wave_adjoint_scaled; needs v != 0 everywhere; the faster on GB300),
    or "auto" (mu where every interior m > 0, else lam).
    """

    def __init__(self, nx, ny, nz, src, rec_z, h, dt, sponge_width=20, sponge_a=0.015, r=4,
                 coeffs=None, device="cuda", adjoint="auto"):
        if adjoint not in ("lam", "mu", "auto"):
            raise ValueError("adjoint is 'lam', 'mu' or 'auto'")
        self.adjoint = adjoint
        self.nx, self.ny, self.nz, self.r = int(nx), int(ny), int(nz), int(r)
        self.src = np.asarray(src, np.int32).reshape(-1, 3)
        self.nshots = len(self.src)
        self.rec_z, self.h, self.dt = int(rec_z), float(h), float(dt)
        self.device = torch.device(device)
        if coeffs is None:
            if self.r != 4:
                raise ValueError("default weights are the radius-4 FD8 set")
            fd8 = (-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)
            row = [fd8[abs(d)] for d in range(-4, 5)]
            coeffs = np.array([row] * 3, np.float32)
        self.coeffs = np.ascontiguousarray(np.asarray(coeffs, np.float32))
        self.m = _lib.padded_empty(nx, ny, nz, r, device=self.device)
        self.p = [_lib.padded_empty(nx, ny, nz, r, nshots=self.nshots, device=self.device)
                  for _ in range(2)]
        py, pz, ss = _lib.field_geometry(self.p[0])
        self.pitch = (py, pz, ss)
        self.desc, self._src_keep = _lib.wave_desc(nx, ny, nz, r, self.nshots, py, pz, ss,
                                                   sponge_width, sponge_a, self.rec_z, self.src)
        self.field_elems = self.p[0].untyped_storage().nbytes() // 4

    # ------------------------------------------------------------- helpers
    def new_fields(self, zero=True):
        return _lib.padded_empty(self.nx, self.ny, self.nz, self.r, nshots=self.nshots,
                                 device=self.device, zero=zero)

    def flat(self, f):
        return torch.as_strided(f, (f.untyped_storage().nbytes() // 4,), (1,), 0)

    def set_velocity(self, v):
        v = v.detach().to(self.device, torch.float32).contiguous()
        _lib.model_from_velocity(self.desc, v, self.m, self.dt, self.h)
        return v

    def n_checkpoints(self, nsteps, every):
        return (nsteps + every - 1) // every

    # ------------------------------------------------------------- forward
    def forward(self, v, amps, nsteps, ckpt_every=0, graph=False):
        """Run nsteps steps from rest; returns records (nsteps, nshots, ny, nx)
        and, when ckpt_every > 0, the checkpoint buffer
        (n_ckpt, 2, field elements): (a^k, a^{k-1}) at k = j*ckpt_every."""
        self.set_velocity(v)
        for f in self.p:
            f.zero_()
        amps = amps.to(self.device, torch.float32).contiguous()
        rec = torch.empty((nsteps, self.nshots, self.ny, self.nx), device=self.device)
        ckpt = None
        if ckpt_every:
            ckpt = torch.empty((self.n_checkpoints(nsteps, ckpt_every), 2, self.field_elems),
                               device=self.device)
        _lib.wave_forward(self.desc, self.coeffs, self.m, amps, nsteps, self.p[0], self.p[1], rec,
                          ckpt, ckpt_every, graph=graph)
        return rec, ckpt

    def _view(self, flat):
        """The (nshots, Z, Y, X) field view of a flat field image (e.g. one
        checkpoint slot), starting where the image starts."""
        py, pz, ss = self.pitch
        X = self.nx + 2 * self.r
        return torch.as_strided(flat, (self.nshots, self.nz + 2 * self.r, self.ny + 2 * self.r, X),
                                (ss, pz, py, 1), flat.storage_offset())

    # ------------------------------------------------------------ gradient
    def gradient_m(self, amps, resid, ckpt, ckpt_every, deterministic=False, scaled=None):
        """dJ/dm (FP64, (nz, ny, nx)) for records whose residual is ``resid``
        (nsteps, nshots, ny, nx), from the forward checkpoints; the velocity
        (model m) must be the one the checkpoints were made with.

        Each segment is recomputed out of place from the checkpoint images
        themselves (no copies), keeping L a^n of every step for the adjoint
        steps (mms_wave_step_lap / mms_wave_adjoint_lap).  The shots add their terms
        to one FP64 gradient with atomics, whose order varies from run to
        run; ``deterministic`` gives every shot its own FP64 slice (plain
        read-modify-write, summed once at the end) for bit-reproducible
        results, at about 15 % more adjoint time with two shots.  ``scaled``
        carries the adjoint state as mu = m G lam (mms_wave_adjoint_scaled;
        needs m > 0 at every interior point) instead of lam; None takes the
        propagator's ``adjoint`` setting.  The same gradient either way."""
        nsteps = resid.shape[0]
        resid = resid.to(self.device, torch.float32).contiguous()
        amps = amps.to(self.device, torch.float32).contiguous()
        npts = self.nz * self.ny * self.nx
        per_shot = deterministic and self.nshots > 1
        grad = torch.zeros(((self.nshots,) if per_shot else ()) + (self.nz, self.ny, self.nx),
                           device=self.device, dtype=torch.float64)
        desc_g = self.desc
        if per_shot:
            py, pz, ss = self.pitch
            desc_g, self._src_keep_g = _lib.wave_desc(self.nx, self.ny, self.nz, self.r, self.nshots, py,
                                                      pz, ss, self.desc.sponge_width, self.desc.sponge_a,
                                                      self.rec_z, self.src, grad_shot_stride=npts)
        # The recompute of a segment steps a^{k0} .. a^{k1-1} forward from the
        # checkpoint images (never overwritten) through two scratch fields and
        # keeps what the adjoint needs: lap[i] = L a^{k0+i}, which each step
        # computes anyway.  The adjoint step that forms lam^n adds
        # g lam^{n+1} (L a^n); for n = k1 that is the next segment's lap[0],
        # carried over (for the last segment lam^{Nt+1} = 0: no term).
        scratch = [self.new_fields(zero=True), self.new_fields(zero=True)]
        lap = [self.new_fields() for _ in range(ckpt_every)]
        carry, have_carry = self.new_fields(), False
        # The adjoint states: lam, or (scaled) mu = m G lam, whose step has the
        # forward step's form; the gradient terms are the same.
        r = self.r
        if scaled is None:
            scaled = (self.adjoint == "mu" or
                      (self.adjoint == "auto" and bool((self.m[r:-r, r:-r, r:-r] > 0).all())))
        adjoint = _lib.wave_adjoint_scaled if scaled else _lib.wave_adjoint_lap
        lam = [self.new_fields(), self.new_fields()]   # lam^{n+2}, lam^{n+1} (or mu)
        nseg = self.n_checkpoints(nsteps, ckpt_every)
        for j in range(nseg - 1, -1, -1):
            k0 = j * ckpt_every
            k1 = min(k0 + ckpt_every, nsteps)
            old_f, cur_f = self._view(ckpt[j, 1]), self._view(ckpt[j, 0])
            for n in range(k0, k1):
                # out of place; from the third step on, over a^{n-1}
                nxt = scratch[(n - k0) % 2]
                _lib.wave_step_lap(self.desc, self.coeffs, self.m, cur_f, old_f, nxt, lap[n - k0], amps[n])
                old_f, cur_f = cur_f, nxt
            for n in range(k1, k0, -1):                   # lam^n, n = k1 .. k0+1
                la = lap[n - k0] if n < k1 else (carry if have_carry else None)
                adjoint(desc_g, self.coeffs, self.m, lam[1], lam[0], resid[n - 1], la, grad)
                lam[0], lam[1] = lam[1], lam[0]
            lap[0], carry = carry, lap[0]
            have_carry = True
        if per_shot:
            _lib.sum_f64(grad, grad[0])
            grad = grad[0]
        if scaled:   # the sum of mu^{n+1} (L a^n) is m dJ/dm
            _lib.grad_divide_m(self.desc, self.m, grad)
        return grad

    def gradient_v(self, v, grad_m):
        v = v.detach().to(self.device, torch.float32).contiguous()
        gv = torch.empty_like(grad_m)
        _lib.grad_to_velocity(grad_m, v, gv, self.dt, self.h)
        return gv


class WaveFunction(torch.autograd.Function):
    """records = WaveFunction.apply(v, prop, amps, nsteps, ckpt_every)."""

    @staticmethod
    def forward(ctx, v, prop: WavePropagator, amps, nsteps: int, ckpt_every: int = 20):
        rec, ckpt = prop.forward(v, amps, nsteps, ckpt_every=ckpt_every)
        ctx.prop, ctx.nsteps, ctx.every = prop, nsteps, ckpt_every
        ctx.save_for_backward(v, amps, ckpt)
        return rec

    @staticmethod
    def backward(ctx, grad_rec):
        v, amps, ckpt = ctx.saved_tensors
        prop = ctx.prop
        prop.set_velocity(v)
        gm = prop.gradient_m(amps, grad_rec, ckpt, ctx.every)
        gv = prop.gradient_v(v, gm)
        return gv.to(v.dtype), None, None, None, None
