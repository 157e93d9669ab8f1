#!/usr/bin/env python3
"""Throughput of the box-stencil sweeps on GB300: GPoints/s and roofline.

Workload (one step): one radius-1 (27-point) and one radius-2 (125-point) box
sweep of a 512^3 FP32 interior plus halo, coefficients ~ N(0, 1/npts), input
U[-1, 1], through the library's AUTO path (the fastest path that meets FP32
accuracy).  Inputs (550 MB each) and outputs (537 MB each) exceed the 129 MB
L2, so no flush is needed between steps.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Under torchrun (N > 1) every rank sweeps its own independent grids (weak
scaling, no collective on the data path); `value` counts the points of all
ranks over the slowest rank's time.  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "GPoints/s & % roofline per sweep; TC split-precision vs FP32 CUDA-core at ≤1e-5"
N = 512
RADII = (1, 2)
FLOP_PER_PT = {1: 2 * 27, 2: 2 * 125}
WORKLOAD = "box stencil sweeps r=1 (27 pt) + r=2 (125 pt), 512^3 FP32 interior + halo"

# Sweeps of one step, per workload: (shape, radius, n, coefficient recipe).
WORKLOADS = {
    "box512": [("box", 1, 512), ("box", 2, 512)],
    "star1024": [("star", 4, 1024)],
    "star512": [("star", 4, 512)],
    "plane8192": [("star2d", 2, 8192), ("star2d", 4, 8192), ("box2d", 2, 8192), ("box2d", 3, 8192)],
    "rtm512": None,    # acoustic forward: 8 shots x 512^3, 500 steps (see run_wave)
    "grad256": None,   # adjoint gradient: 2 shots x 256^3, 200 steps, checkpoint 20
    "vti512": None,    # VTI forward: 4 shots x 512^3 (see run_aniso)
    "tti512": None,    # TTI forward: 2 shots x 512^3 (see run_aniso)
    "fp64_512": [("star", 4, 512), ("box", 1, 512)],   # FP64 sweeps (see run_f64)
}
WORKLOAD_NAMES = {
    "box512": WORKLOAD,
    "star1024": "star stencil sweep r=4 (25 pt, FD8 weights), 1024^3 FP32 interior + halo, "
                "16 sinusoids + 1e-3 noise",
    "star512": "star stencil sweep r=4 (25 pt, FD8 weights), 512^3 FP32 interior + halo, "
               "16 sinusoids + 1e-3 noise (profiling size)",
    "plane8192": "Table I's 2D kernels (2DStarR2, 2DStarR4, 2DBoxR2, 2DBoxR3) on one 8192^2 FP32 plane "
                 "each, weights N(0, 1/npts), input U[-1, 1]",
    "rtm512": "batched acoustic forward, 8 shots x 512^3, r=4 FD8 star, 20-cell sponge, h=10 m, "
              "CFL 0.4, 15 Hz Ricker, one CUDA graph per run",
    "grad256": "adjoint gradient of 0.5|d - d_obs|^2 wrt velocity, 2 shots x 256^3, 200 steps, "
               "checkpoint every 20 with recompute, FP64 accumulation",
    "vti512": "VTI forward (sigma_H, sigma_V of Sec. 2.1), 4 shots x 512^3, r=4 FD8 star, layered vp with "
              "per-layer eps, delta, 20-cell sponge, h=10 m, CFL 0.4, 15 Hz Ricker",
    "tti512": "TTI forward (p, q with H1, H2 of Sec. 2.1), 2 shots x 512^3, r=4 FD8 second- and first-derivative "
              "weights, layered vp with per-layer eps, delta, vs = vp/2, alpha = 1, smooth tilt, 20-cell sponge",
}
WORKLOAD_NAMES["fp64_512"] = ("FP64 sweeps: star r=4 (FD8 weights) and box r=1 (weights N(0, 1/27)), 512^3 "
                              "FP64 interior + halo, input U[-1, 1]")
ANISO = {"vti512": dict(kind="vti", n=512, shots=4, bytes_per_point_step=32,
                        kernel="vti_fwd_kernel (two coupled r=4 stars + leapfrog + sponge + source + receivers)"),
         # per point-step: the p pass (read p and the tilt, 16 B; write Lap p
         # and H1 p, 8 B) and the q pass with the combine fused in (read q,
         # Lap p, H1 p, the 8 medium fields, p^n, p^{n-1}, q^{n-1}: 56 B;
         # write p^{n+1}, q^{n+1}: 8 B)
         "tti512": dict(kind="tti", n=512, shots=2, bytes_per_point_step=88,
                        kernel="whole step: tti_deriv_kernel<p> + tti_deriv_kernel<q, combine fused>")}


def sweep_coeffs(shape, r):
    if shape == "star":
        return workloads.star_coeffs(r)
    if shape in PLANAR:
        return workloads.normal_coeffs(shape, r, workload=6, salt=r)
    return workloads.normal_coeffs("box", r, workload=2, salt=r)


PLANAR = ("star2d", "box2d")


def sweep_dims(shape, n):
    """Interior (nx, ny, nz) of a sweep of size n: n^3, or one n^2 plane."""
    return (n, n, 1) if shape in PLANAR else (n, n, n)


def sweep_points(shape, n):
    nx, ny, nz = sweep_dims(shape, n)
    return nx * ny * nz


def sweep_bytes(shape, r, n):
    """Algorithmic bytes: the padded input read once, the output written once."""
    nx, ny, nz = sweep_dims(shape, n)
    rz = 0 if shape in PLANAR else r
    return 4 * ((nx + 2 * r) * (ny + 2 * r) * (nz + 2 * rz) + nx * ny * nz)


def sweep_input(shape, r, n, rank):
    if shape in PLANAR:
        return workloads.uniform_grid2d(n, n, 1, r, workload=6, salt=r + 100 * rank)
    if shape == "star":
        return workloads.sinusoid_grid(n, n, n, r, workload=3, salt=rank)
    return workloads.uniform_grid(n, n, n, r, workload=2, salt=r + 100 * rank)


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's x (x itself without a process group):
    the job's time is its slowest rank's."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput in G units per second: every rank processes
    units_per_rank (weak scaling) in `seconds` (the slowest rank's time)."""
    return world * units_per_rank / seconds / 1e9


def flop_per_pt(shape, r):
    return 2 * workloads.n_points(shape, r)


ERROR_NOTE = ("max |result - oracle| / max |oracle| at seeded sample points (corners and face centres "
              "included) of the timed run's own inputs, against the FP64 oracle; wave, VTI and TTI: one step "
              "after the timed steps, from the state they left, shot 0")


def rel_err(got, ref) -> float:
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def sweep_error(shape, r, coeffs, host_grid, out, salt=0, npts=2000) -> float:
    """Max-relative error of a sweep's output `out` (device or host, (nz, ny,
    nx)) against the FP64 oracle on the padded host input `host_grid`."""
    import oracle
    nz, ny, nx = out.shape
    pts = workloads.sample_points(nx, ny, nz, npts, workload=9, salt=salt)
    if shape in PLANAR:
        ref = oracle.stencil2d_points(shape, r, coeffs, host_grid, pts)
    else:
        ref = oracle.stencil_points(shape, r, coeffs, host_grid, pts)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    if not isinstance(out, np.ndarray):            # a torch tensor on the device
        import torch
        idx = torch.from_numpy(pts).to(out.device)
        got = out[idx[:, 2], idx[:, 1], idx[:, 0]].double().cpu().numpy()
    else:
        got = np.asarray(out)[z, y, x]
    return rel_err(got, ref)


def at_points(pts, shape, values):
    """A zero FP64 array of `shape` holding `values` at the points (x, y, z)
    (np.zeros leaves untouched pages unallocated): the oracle's point-wise
    steps read a per-point medium only at their points."""
    a = np.zeros(shape)
    a[pts[:, 2], pts[:, 1], pts[:, 0]] = values
    return a


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 1900.0, 2070.0, "fallback"


def bf16_sustained_peak():
    """Measured BF16 dense peak of a seconds-long GEMM loop (the timed region
    here is one), else the fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if "bf16_tflops_sustained" in d:
            return d["bf16_tflops_sustained"], "measured sustained"
    return 1700.0, "fallback sustained"


def captured_traffic(key: str, points: int):
    """DRAM bytes of one launch from the committed ncu capture of this kernel
    (profiles/traffic.json), scaled by points; None when the kernel's sources
    changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(key)
    if not rec:
        return None
    for f, h in rec["sources"].items():
        path = os.path.join(ROOT, "paper_2507_11067_gb300", "csrc", f)
        if not os.path.exists(path) or code_hash(path) != h:
            return None
    return rec["dram_bytes_per_point"] * points


def code_hash(path: str) -> str:
    """Hash of a CUDA source without its comments and blank lines: the
    kernel the counters were taken on, whatever its comments say."""
    import hashlib
    import re
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    code = "\n".join(l.rstrip() for l in text.splitlines() if l.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


TC_PATHS = ("tf32", "3xtf32", "bf16x3")


def tc_dense_flop_per_pt(path: str, r: int, planar: bool = False) -> float:
    """Dense work the banded MMAs issue per output point (band zeros
    included).  A tile of the tensor-core kernel is 4 x-subtiles of
    TXO = 16 - 2r (rounded down to a multiple of 4) outputs by TY = 32 - 2r
    rows; per output plane it runs, for
    each plane the stencil reaches in z ((2r+1) for the box, 1 for planar
    stencils and the star's in-plane part), M = 128 lanes x N = (2r+1) TXO
    (rounded up to 16) x K = 16 MMAs, times the split products (3 for
    3xTF32 / BF16x3, 1 for TF32)."""
    txo, ty, w = (16 - 2 * r) & ~3, 32 - 2 * r, 2 * r + 1
    n = -(-w * txo // 16) * 16
    planes = 1 if planar else w
    prods = 1 if path == "tf32" else 3
    return 2.0 * 128 * n * 16 * planes * prods / (4 * txo * ty)


def tc_roofline(shape: str, r: int, path: str, npts: int, bytes_alg: float, sec: float,
                hbm_peak: float, bf16_peak: float, bf16_src: str) -> dict:
    """Roofline of a tensor-core sweep on the stencil's own work: the slower
    of its two floors, the algorithmic HBM bytes against the measured copy
    bandwidth and its useful 2 flop per coefficient against the tensor peak
    (BF16's; TF32 at the nominal ratio 1.1/2.25).  The banded MMAs' dense
    work (band zeros and split products included) and its fraction of the
    tensor peak go beside it."""
    planar = shape in PLANAR
    tpk = bf16_peak if path == "bf16x3" else bf16_peak * 1.1 / 2.25
    useful = flop_per_pt(shape, r) * npts
    dense = tc_dense_flop_per_pt(path, r, planar or shape == "star") * npts
    t_hbm = bytes_alg / (hbm_peak * 1e9)
    t_tc = useful / (tpk * 1e12)
    if t_hbm >= t_tc:
        roof = {"bound": "hbm", "achieved": bytes_alg / sec / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": bytes_alg / sec / 1e9 / hbm_peak}
    else:
        roof = {"bound": "tensor", "achieved": useful / sec / 1e12, "peak": tpk, "unit": "TFLOP/s",
                "frac": useful / sec / 1e12 / tpk}
    roof["dense_tflops"] = dense / sec / 1e12
    roof["tensor_pipe_frac"] = dense / sec / 1e12 / tpk
    roof["peak_note"] = (f"bound = the slower floor of the stencil's own work: {bytes_alg / npts:.2f} B/pt over "
                         f"MEASURED_PEAKS.json hbm_gbs, {flop_per_pt(shape, r)} flop/pt over bf16 ({bf16_src}"
                         f"{'' if path == 'bf16x3' else ' x 1.1/2.25 (TF32)'}); dense_tflops counts the banded "
                         f"MMAs' {tc_dense_flop_per_pt(path, r, planar or shape == 'star'):.0f} flop/pt "
                         f"(band zeros and split products included)")
    return roof


def fp32_alu_peak_tflops(n_sm: int, mhz: float) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flop) per lane per clock.
    return n_sm * 128 * 2 * mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs; the raw
    samples go to $MMS_CLOCKS_DIR (default: the system temp directory)."""

    def __init__(self, gpu_index: int):
        import tempfile
        self.p = None
        folder = os.environ.get("MMS_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, f"clocks_bench_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(planes: int, salt: int = 0, plan=None):
    """Oracle on the first `planes` output planes of every sweep of the plan
    (default: the box workload's two sweeps), on seeded slabs of the same
    sizes and value distributions; returns (points, seconds, threads)."""
    import oracle
    plan = plan or WORKLOADS["box512"]
    pts, secs = 0, 0.0
    for shape, r, n in plan:
        c = sweep_coeffs(shape, r)
        g = workloads.rng(2 if shape == "box" else 3, 50 + r + 100 * salt)
        if shape in PLANAR:
            # a slab of `planes` output rows of the n^2 plane
            sub = g.uniform(-1, 1, size=(1, planes + 2 * r, n + 2 * r))
            t0 = time.perf_counter()
            oracle.stencil2d(shape, r, c, sub)
            secs += time.perf_counter() - t0
            pts += planes * n
            continue
        sub = g.uniform(-1, 1, size=(planes + 2 * r, n + 2 * r, n + 2 * r))
        t0 = time.perf_counter()
        oracle.stencil(shape, r, c, sub)
        secs += time.perf_counter() - t0
        pts += planes * n * n
    return pts, secs, oracle_threads()


def oracle_wave_sample(planes: int, n: int, gradient: bool, salt: int = 0):
    """Oracle wave steps on a slab of `planes` z-planes of one n x n shot:
    one forward step, or for the gradient workload the forward step, its
    recomputation and the adjoint step with the gradient term (the work of
    one point-step of the gradient); returns (point-steps, seconds, threads)."""
    import oracle
    r = 4
    g = workloads.rng(4, 80 + 100 * salt)
    v = g.uniform(1500.0, 4500.0, size=(planes, n, n))
    dt, h = 0.4 * 10.0 / 4500.0, 10.0
    prob = oracle.WaveProblem(r, workloads.fd8_star_coeffs(), oracle.model_m(v, dt, h), (20, 0.015),
                              [(n // 2, n // 2, planes // 2)], np.full((2, 1), 1e-3), 0)
    a_cur, a_prev = (oracle.pad(g.uniform(-1, 1, (planes, n, n)), r) for _ in range(2))
    t0 = time.perf_counter()
    nxt = prob.step(a_cur, a_prev, 0, 1)
    if gradient:
        prob.step(a_cur, a_prev, 0, 1)
        grad = np.zeros((planes, n, n))
        prob.adjoint_step(nxt, a_cur, None, a_prev, grad)
    secs = time.perf_counter() - t0
    return planes * n * n, secs, oracle_threads()


def oracle_aniso_sample(planes: int, n: int, kind: str, salt: int = 0):
    """One FP64 oracle step of the anisotropic workload on a slab of `planes`
    z-planes of one n x n shot; returns (point-steps, seconds, threads)."""
    from oracle import aniso
    r = 4
    tti = kind == "tti"
    a = workloads.AnisoInputs(n, n, planes, 1, 2, workload=7 if tti else 6, noise=False, salt=80 + salt, tti=tti)
    g = workloads.rng(6, 90 + salt)
    fields = [oracle_pad(g.uniform(-1, 1, (planes, n, n)), r) for _ in range(4)]
    if tti:
        med = aniso.tti_medium(a.vp, a.vs, a.eps, a.delta, a.alpha, a.dt, a.h)
        tilt = aniso.tilt_axis(a.theta, a.phi)
        t0 = time.perf_counter()
        aniso.tti_step(r, med, tilt, (20, 0.015), a.src[0], 1e-3, *fields)
    else:
        mh, mv = aniso.vti_medium(a.vp, a.eps, a.delta, a.dt, a.h)
        t0 = time.perf_counter()
        aniso.vti_step(r, workloads.fd8_star_coeffs(), mh, mv, (20, 0.015), a.src[0], 1e-3, *fields)
    secs = time.perf_counter() - t0
    return planes * n * n, secs, oracle_threads()


def oracle_pad(f, r):
    import oracle
    return oracle.pad(f, r)


def cpu_baseline(sample, unit, what, budget_s=5.0):
    """The oracle timed on the host: on all cores (OpenMP), then on one core,
    each on a slab sized for about budget_s seconds; `what` names the sample
    ({planes} is filled in)."""
    import oracle
    oracle.build()
    planes = calibrate_planes(budget_s, sample)
    p, secs, threads = sample(planes)
    out = {"value": p / secs / 1e9, "unit": unit, "cores": threads, "kind": "oracle",
           "sample": what.format(planes=planes)}
    old = oracle.set_threads(1)
    try:
        planes1 = calibrate_planes(budget_s, sample)
        p, secs, _ = sample(planes1)
    finally:
        oracle.set_threads(old)
    out["one_core"] = {"value": p / secs / 1e9, "unit": unit, "cores": 1, "sample": what.format(planes=planes1)}
    return out


def oracle_threads() -> int:
    import oracle
    return oracle.set_threads(0)


def calibrate_planes(budget_s: float, sample=None) -> int:
    sample = sample or (lambda planes, salt=0: oracle_sample(planes, salt))
    pts, secs, _ = sample(2)
    per_plane = secs / 2
    return max(2, min(512, int(budget_s / max(per_plane, 1e-6))))


def run_reference(args):
    """The base contract's reference arm: the FP64 oracle as it stands, on the
    host cores, timed on bounded samples of the selected workload (each step
    about MMS_REF_STEP_SECONDS of CPU work)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    budget = float(os.environ.get("MMS_REF_STEP_SECONDS", "6"))
    if args.workload in ("rtm512", "grad256"):
        n = 512 if args.workload == "rtm512" else 256
        grad = args.workload == "grad256"

        def sample(planes, salt=0):
            return oracle_wave_sample(planes, n, grad, salt)
        unit = "GPoint-steps/s"
        what = ("forward step" if not grad else "forward step, its recomputation and the adjoint step")
    elif args.workload in ANISO:
        spec = ANISO[args.workload]

        def sample(planes, salt=0):
            return oracle_aniso_sample(planes, spec["n"], spec["kind"], salt)
        unit = "GPoint-steps/s"
        what = f"{spec['kind'].upper()} step"
    else:
        plan = WORKLOADS[args.workload]

        def sample(planes, salt=0):
            return oracle_sample(planes, salt, plan)
        unit = "GPoints/s"
        what = ", ".join(f"{sh} r={r} {nn}^{2 if sh in PLANAR else 3}" for sh, r, nn in plan)
    planes = calibrate_planes(budget, sample)
    for _ in range(args.warmup):
        sample(max(2, planes // 8))
    total_pts, total_s = 0, 0.0
    threads = 1
    args.steps = args.steps or 3
    for k in range(args.steps):
        p, secs, threads = sample(planes, salt=k)
        total_pts += p
        total_s += secs
    value = total_pts / total_s / 1e9
    sample_txt = f"FP64 oracle ({what}) on a seeded slab of {planes} output planes per sweep, per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES[args.workload], "sample": sample_txt},
        "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
                         "sample": sample_txt},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="0 = about 2 s of timed sweeps")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="box512", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="auto")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=0,
                    help="grid edge (0 = the workload's own; smaller for profiling captures); not for rtm512 or grad256")
    ap.add_argument("--adjoint", default="auto", choices=["auto", "lam", "mu"],
                    help="grad256: the adjoint state, lam or mu = m G lam (auto: mu where m > 0 everywhere)")
    ap.add_argument("--shots", type=int, default=0,
                    help="shots of the wave workloads (0 = the workload's own: 8 for rtm512, 2 for grad256)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("rtm512", "grad256"):
        return run_wave(args)
    if args.workload in ANISO:
        return run_aniso(args)
    if args.workload == "fp64_512":
        return run_f64(args)

    import torch
    import paper_2507_11067_gb300 as mms

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mms.build()
    mms.load()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    hbm_peak, bf16_peak, sm_max_mhz, peak_src = peaks()

    # ---- inputs (seeded per rank), resident in HBM before timing
    from paper_2507_11067_gb300 import tune
    tune.load_table()
    plan = WORKLOADS[args.workload]
    if args.n:   # a smaller grid of the same sweeps (profiling captures)
        plan = [(shape, r, args.n) for shape, r, _ in plan]
    coeffs, inputs, outputs, hosts, host_out, grids = [], [], [], [], [], []
    for (shape, r, n) in plan:
        coeffs.append(sweep_coeffs(shape, r))
        grid = sweep_input(shape, r, n, rank)
        grids.append(grid)
        nx_, ny_, nz_ = sweep_dims(shape, n)
        alloc = mms.padded_empty2d if shape in PLANAR else mms.padded_empty
        # host buffer pinned with the device pitch, so each copy is one memcpy
        hp = alloc(nx_, ny_, nz_, r, device="cpu", zero=False)
        hp = torch.as_strided(torch.empty(hp.untyped_storage().nbytes() // 4, pin_memory=True),
                              hp.shape, hp.stride())
        hp.copy_(torch.from_numpy(grid))
        hosts.append(hp)
        inputs.append(alloc(nx_, ny_, nz_, r, device=dev, zero=False))
        inputs[-1].copy_(hosts[-1])
        outputs.append(torch.empty((nz_, ny_, nx_), device=dev))
        host_out.append(torch.empty((nz_, ny_, nx_), pin_memory=True))
    stream = torch.cuda.current_stream(dev)
    steps = args.steps or max(20, int(2000 / max(1, sum(sweep_points(sh, n) for sh, _, n in plan) / 2.7e8)))

    def sweep(i):
        shape, r, _ = plan[i]
        mms.apply(shape, r, coeffs[i], inputs[i], outputs[i], path=args.path)

    # ---- device-resident timing
    for _ in range(args.warmup):
        for i in range(len(plan)):
            sweep(i)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    kernel_ev = [[] for _ in plan]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(steps):
        for i in range(len(plan)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sweep(i)
            b.record(stream)
            kernel_ev[i].append((a, b))
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed = max_over_ranks(t_start.elapsed_time(t_end) / 1e3, dist, dev)
    pts_step = sum(sweep_points(sh, n) for sh, _, n in plan)
    value = job_rate(world, pts_step * steps, elapsed)
    kms = [statistics.mean(a.elapsed_time(b) for a, b in ev) for ev in kernel_ev]

    # ---- end to end through the C ABI with host buffers: every step sweeps
    # the pinned host inputs into pinned host outputs with
    # mms_stencil_apply_host (the library streams z-slabs through the device:
    # copy in, sweep, copy out, pipelined).  Consecutive steps alternate
    # between two streams, so one step's slab pipeline overlaps the next's.
    streams = [stream, torch.cuda.Stream(dev)]
    hout_sets = [host_out, [torch.empty(o.shape, pin_memory=True) for o in host_out]]

    def e2e_step(k):
        st = streams[k % 2]
        for i in range(len(plan)):
            shape, r, _ = plan[i]
            mms.apply_host(shape, r, coeffs[i], hosts[i], hout_sets[k % 2][i], path=args.path, stream=st)

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e_s, e_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(4, min(50, steps // 4))
    e_s.record(streams[0])
    streams[1].wait_event(e_s)
    for k in range(e2e_steps):
        e2e_step(k)
    streams[0].wait_stream(streams[1])
    e_e.record(streams[0])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_s = max_over_ranks(e_s.elapsed_time(e_e) / 1e3, dist, dev)
    h2d = sum(h.untyped_storage().nbytes() for h in hosts)
    d2h = sum(h.numel() * 4 for h in host_out)
    e2e_value = job_rate(world, pts_step * e2e_steps, e2e_s)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # ---- dominant kernel roofline
    path_used = args.path
    alu_peak = fp32_alu_peak_tflops(n_sm, sm_max_mhz)
    di = max(range(len(plan)), key=lambda i: kms[i])
    shape, r, n = plan[di]
    sec = kms[di] / 1e3
    npts = sweep_points(shape, n)
    bytes_alg = sweep_bytes(shape, r, n)
    flops = flop_per_pt(shape, r) * npts
    resolved = mms.auto_path(shape, r) if path_used == "auto" else path_used
    if resolved in TC_PATHS:
        tpk, tsrc = bf16_sustained_peak()
        roofline = tc_roofline(shape, r, resolved, npts, bytes_alg, sec, hbm_peak, tpk, tsrc)
    elif flops / bytes_alg > alu_peak * 1e12 / (hbm_peak * 1e9):
        roofline = {"bound": "alu", "achieved": flops / sec / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": flops / sec / 1e12 / alu_peak, "traffic": None,
                    "peak_note": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {sm_max_mhz:.0f} MHz "
                                 "(max SM clock)"}
    else:
        roofline = {"bound": "hbm", "achieved": bytes_alg / sec / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": bytes_alg / sec / 1e9 / hbm_peak, "traffic": None,
                    "peak_note": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}
    var = mms.default_variant(shape, r, resolved, *sweep_dims(shape, n))
    roofline["kernel"] = f"{shape} r={r} {n}^{2 if shape in PLANAR else 3} sweep ({resolved}, variant {var})"
    roofline["ms"] = kms[di]
    tr = captured_traffic(f"{resolved} {shape} r={r} v{var}", npts)
    roofline["traffic"] = tr
    if tr:
        roofline["traffic_over_algorithmic"] = tr / bytes_alg

    sweeps = {}
    for i, (shape, r, n) in enumerate(plan):
        sec = kms[i] / 1e3
        b = sweep_bytes(shape, r, n)
        f = flop_per_pt(shape, r) * sweep_points(shape, n)
        sweeps[f"{shape}_r{r}_{n}"] = {"ms": kms[i], "gpts": sweep_points(shape, n) / sec / 1e9,
                                       "hbm_gbs": b / sec / 1e9, "hbm_frac": b / sec / 1e9 / hbm_peak,
                                       "tflops": f / sec / 1e12, "alu_frac": f / sec / 1e12 / alu_peak}

    # ---- accuracy of every timed result (outside the timed regions): the
    # device-resident sweeps and the end-to-end outputs, against the oracle
    errors = {}
    for i, (shape, r, n) in enumerate(plan):
        p_i = mms.auto_path(shape, r) if args.path == "auto" else args.path
        errors[f"{shape}_r{r}_{n}_{p_i}"] = sweep_error(shape, r, coeffs[i], grids[i], outputs[i], salt=i)
        errors[f"{shape}_r{r}_{n}_{p_i}_e2e"] = sweep_error(shape, r, coeffs[i], grids[i],
                                                           hout_sets[0][i].numpy(), salt=10 + i)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(lambda p, salt=0: oracle_sample(p, salt, plan), "GPoints/s",
                           "FP64 oracle, " + ", ".join(f"{sh} r={r}" for sh, r, _ in plan) +
                           ", a seeded slab of {planes} output planes per sweep")

    line = {
        "metric": METRIC, "value": value, "unit": "GPoints/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES[args.workload] + (f" at grid edge {args.n}" if args.n else ""),
                   "path": path_used,
                   "sweeps": [f"{sh} r={r} {n}^{2 if sh in PLANAR else 3}" for sh, r, n in plan],
                   "l2": "inputs and outputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "GPoints/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "note": "mms_stencil_apply_host on pinned host grids each step (z-slabs copied in, "
                        "swept and copied out by the library, pipelined); consecutive steps on two "
                        "streams"},
        "gpu_launches": len(plan) * steps,
        "clocks": clk, "peaks": {"hbm_gbs": hbm_peak, "bf16_tflops": bf16_peak, "source": peak_src},
        "sweeps": sweeps, "errors": errors, "error_note": ERROR_NOTE,
    }
    if not args.no_extras:
        line["extras"] = extras(mms, torch, dev, hbm_peak, alu_peak)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_wave(args):
    """The acoustic workloads on one GPU (shots are independent: under
    torchrun each rank runs its own shots, weak scaling)."""
    import torch
    import paper_2507_11067_gb300 as mms
    from paper_2507_11067_gb300.wave import WaveFunction, WavePropagator
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mms.build()
    mms.load()
    hbm_peak, _, _, peak_src = peaks()
    if args.workload == "rtm512":
        n, nshots, nsteps, every = 512, 8, 500, 0
    else:
        n, nshots, nsteps, every = 256, 2, 200, 20
    nshots = args.shots or nshots
    wi = workloads.WaveInputs(n, n, n, nshots=nshots, nsteps=nsteps, workload=4 if n == 512 else 5,
                              noise=True, salt=rank)
    prop = WavePropagator(n, n, n, wi.src, wi.zrec, wi.h, wi.dt, sponge_width=wi.sponge,
                          sponge_a=wi.sponge_a, device=dev, adjoint=args.adjoint)
    v_host = torch.from_numpy(wi.v).pin_memory()
    amps_host = torch.from_numpy(wi.amp).pin_memory()
    v = v_host.to(dev)
    amps = amps_host.to(dev)
    stream = torch.cuda.current_stream(dev)

    if args.workload == "rtm512":
        steps = args.steps or nsteps

        def run():
            rec, _ = prop.forward(v, amps[:steps], steps, graph=True)
            return rec
        launches = steps
    else:
        steps = args.steps or 1
        w0 = workloads.WaveInputs(n, n, n, nshots=nshots, nsteps=nsteps, workload=5, noise=False, salt=rank)
        with torch.no_grad():
            obs, _ = prop.forward(v, amps, nsteps)
        v0 = torch.from_numpy(w0.v).to(dev)

        def run():
            vv = v0.clone().requires_grad_(True)
            rec = WaveFunction.apply(vv, prop, amps, nsteps, every)
            loss = 0.5 * ((rec - obs) ** 2).sum()
            loss.backward()
            return vv.grad
        # forward, recompute and adjoint steps, the two velocity-to-model
        # kernels (forward, backward) and the chain rule
        launches = 3 * nsteps + 3

    for _ in range(max(1, args.warmup // 3)):
        run()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 1 if args.workload == "rtm512" else steps
    t0.record(stream)
    for _ in range(reps):
        out = run()
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed = max_over_ranks(t0.elapsed_time(t1) / 1e3, dist, dev)
    pts = nshots * n ** 3
    if args.workload == "rtm512":
        units = world * pts * steps
        bytes_alg = 16.0 * pts * steps
        # end to end: velocity and wavelet in from pinned host memory, records out
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vv = v_host.to(dev, non_blocking=True)
        aa = amps_host.to(dev, non_blocking=True)
        rec, _ = prop.forward(vv, aa[:steps], steps, graph=True)
        rec_host = rec.to("cpu")
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
        h2d = v_host.numel() * 4 + amps_host.numel() * 4
        d2h = rec_host.numel() * 4
        value = job_rate(world, pts * steps, elapsed)
        e2e = {"value": job_rate(world, pts * steps, e2e_s), "unit": "GPoint-steps/s",
               "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps}
        roof = {"bound": "hbm", "achieved": bytes_alg / elapsed / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": bytes_alg / elapsed / 1e9 / hbm_peak,
                "traffic": captured_traffic("wave_fwd r=4", pts),
                "kernel": "wave_fwd_kernel (fused star r=4 + leapfrog + sponge + source + receivers)",
                "bytes_per_point_step": 16}
        if roof["traffic"]:
            roof["traffic_over_algorithmic"] = roof["traffic"] / (16.0 * pts)
        unit = "GPoint-steps/s"
    else:
        units = world * pts * nsteps * steps
        value = job_rate(world, pts * nsteps * steps, elapsed)
        # end to end: starting velocity, wavelet and observed records in from
        # pinned host memory, the velocity gradient out, one gradient per step
        v0_host = v0.cpu().pin_memory()
        obs_host = obs.cpu().pin_memory()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vv = v0_host.to(dev, non_blocking=True).requires_grad_(True)
        aa = amps_host.to(dev, non_blocking=True)
        oo = obs_host.to(dev, non_blocking=True)
        rec = WaveFunction.apply(vv, prop, aa, nsteps, every)
        (0.5 * ((rec - oo) ** 2).sum()).backward()
        g_host = vv.grad.to("cpu")
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
        e2e = {"value": job_rate(world, pts * nsteps, e2e_s), "unit": "GPoint-steps/s (forward + gradient)",
               "h2d_bytes_per_step": v0_host.numel() * 4 + amps_host.numel() * 4 + obs_host.numel() * 4,
               "d2h_bytes_per_step": g_host.numel() * g_host.element_size()}
        # per shot-point and step: forward 16 B, recompute 20 B (out of place,
        # no copies; it also writes L a^n), adjoint 20 B (its state at n+1
        # and n+2, m, L a^n read, the state at n written), and the FP64
        # gradient's read-modify-write, 16 B per point shared by the shots
        # (their reductions meet in L2)
        bpp = 56.0 + 16.0 / nshots
        bytes_alg = bpp * pts * nsteps * steps
        ri = prop.r
        mu = args.adjoint == "mu" or (args.adjoint == "auto" and bool((prop.m[ri:-ri, ri:-ri, ri:-ri] > 0).all()))
        roof = {"bound": "hbm", "achieved": bytes_alg / elapsed / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": bytes_alg / elapsed / 1e9 / hbm_peak, "traffic": None,
                "kernel": ("wave_fwd_kernel: forward, recompute writing L a^n, and the adjoint in mu = m G lam "
                           "(one FP64 bulk reduction per output row)") if mu else
                          "wave_fwd_kernel (forward, recompute writing L a^n) + wave_adj_kernel (FP64 atomics)",
                "bytes_per_point_step": bpp}
        unit = "GPoint-steps/s"
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        grad = args.workload == "grad256"
        cpu = cpu_baseline(lambda p, salt=0: oracle_wave_sample(p, n, grad, salt), unit,
                           f"FP64 oracle {'forward, recompute and adjoint steps' if grad else 'forward step'} "
                           f"of one shot on a seeded {{planes}} x {n} x {n} slab")
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / (steps if args.workload == "rtm512" else reps),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": {"workload": WORKLOAD_NAMES[args.workload], "shots": nshots,
                                                "n": n, "time_steps": nsteps if args.workload != "rtm512" else steps,
                                                **({"adjoint": args.adjoint} if args.workload == "grad256" else {})},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches * reps, "clocks": clk,
                "peaks": {"hbm_gbs": hbm_peak, "source": peak_src}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_aniso(args):
    """The anisotropic forward workloads on one GPU: `steps` time steps of all
    shots, one fused launch per step (shots are independent: under torchrun
    each rank runs its own, weak scaling)."""
    import torch
    import paper_2507_11067_gb300 as mms
    spec = ANISO[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mms.build()
    mms.load()
    hbm_peak, _, _, peak_src = peaks()
    n, r = args.n or spec["n"], 4
    nshots = args.shots or spec["shots"]
    steps = args.steps or 200
    tti = spec["kind"] == "tti"
    a = workloads.AnisoInputs(n, n, n, nshots, steps, workload=7 if tti else 6, salt=rank, tti=tti)
    f = [mms.padded_empty(n, n, n, r, device=dev, nshots=nshots) for _ in range(4)]
    py, pz, ss = mms.field_geometry(f[0])
    desc, _src = mms.wave_desc(n, n, n, r, nshots, py, pz, ss, a.wave.sponge, a.wave.sponge_a, a.zrec, a.src)
    if tti:
        host_in = [torch.from_numpy(x).pin_memory() for x in (a.vp, a.vs, a.eps, a.delta, a.alpha, a.theta, a.phi)]
        med = [torch.empty((8, n, n, n), device=dev)]
        work = torch.empty((4, nshots, n, n, n), device=dev)
        w2, w1 = workloads.fd8_rows()
    else:
        host_in = [torch.from_numpy(x).pin_memory() for x in (a.vp, a.eps, a.delta)]
        med = [mms.padded_empty(n, n, n, r, device=dev) for _ in range(2)]
        cf = workloads.fd8_star_coeffs()
    amps_host = torch.from_numpy(a.amp).pin_memory()
    stream = torch.cuda.current_stream(dev)
    rec = torch.zeros((steps, nshots, n, n), device=dev)

    def run(k, inputs, amps, record=True):
        if inputs is not None:
            if tti:
                mms.tti_model(desc, *inputs, med[0], a.dt, a.h)
            else:
                mms.vti_model(desc, *inputs, med[0], med[1], a.dt, a.h)
            for x in f:
                x.zero_()
        cur = list(f)
        for i in range(k):
            if tti:
                mms.tti_step(desc, w2, w1, med[0], cur[0], cur[1], cur[2], cur[3], cur[2], cur[3], work, amps[i],
                             rec[i] if record else None)
            else:
                mms.vti_step(desc, cf, med[0], med[1], cur[0], cur[1], cur[2], cur[3], cur[2], cur[3], amps[i],
                             rec[i] if record else None)
            cur = [cur[2], cur[3], cur[0], cur[1]]
        return cur

    dev_in = [x.to(dev) for x in host_in]
    amps = amps_host.to(dev)
    run(0, dev_in, amps)
    for _ in range(args.warmup):
        run(1, None, amps)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    run(steps, None, amps)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed = max_over_ranks(t0.elapsed_time(t1) / 1e3, dist, dev)
    pts = nshots * n ** 3
    bpp = spec["bytes_per_point_step"]
    bytes_alg = float(bpp) * pts * steps
    # end to end: the medium and the wavelet in from pinned host memory, the
    # model kernel, the steps with receivers, the records out
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ins = [x.to(dev, non_blocking=True) for x in host_in]
    aa = amps_host.to(dev, non_blocking=True)
    run(steps, ins, aa)
    rec_host = rec.to("cpu")
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
    h2d = sum(x.numel() * 4 for x in host_in) + amps_host.numel() * 4
    d2h = rec_host.numel() * 4
    value = job_rate(world, pts * steps, elapsed)
    e2e = {"value": job_rate(world, pts * steps, e2e_s), "unit": "GPoint-steps/s",
           "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps}
    key = f"{spec['kind']}_fwd r=4"
    roof = {"bound": "hbm", "achieved": bytes_alg / elapsed / 1e9, "peak": hbm_peak, "unit": "GB/s",
            "frac": bytes_alg / elapsed / 1e9 / hbm_peak, "traffic": captured_traffic(key, nshots * n ** 3),
            "kernel": spec["kernel"], "bytes_per_point_step": bpp}
    if roof["traffic"]:
        roof["traffic_over_algorithmic"] = roof["traffic"] / (float(bpp) * pts)
    unit = "GPoint-steps/s"
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(lambda p, salt=0: oracle_aniso_sample(p, n, spec["kind"], salt), unit,
                           f"FP64 oracle {spec['kind'].upper()} step of one shot on a seeded {{planes}} x {n} x {n} "
                           "slab")
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD_NAMES[args.workload], "shots": nshots, "n": n,
                           "time_steps": steps, "l2": "inputs larger than L2"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": steps * (2 if tti else 1), "clocks": clk,
                "peaks": {"hbm_gbs": hbm_peak, "source": peak_src}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_f64(args):
    """FP64 sweeps on one GPU (independent grids per rank, weak scaling):
    bound by the FP64 pipe, reported against its peak."""
    import torch
    import paper_2507_11067_gb300 as mms
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mms.build()
    mms.load()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    hbm_peak, _, sm_max_mhz, peak_src = peaks()
    plan = WORKLOADS[args.workload]
    coeffs, ins, outs, hosts, houts = [], [], [], [], []
    for shape, r, n in plan:
        coeffs.append(np.asarray(sweep_coeffs(shape, r), np.float64))
        grid = sweep_input(shape, r, n, rank)
        d = mms.padded_empty(n, n, n, r, device=dev, dtype=torch.float64, zero=False)
        h = torch.empty(d.shape, dtype=torch.float64, pin_memory=True)
        h.copy_(torch.from_numpy(grid))
        d.copy_(h)
        del grid
        ins.append(d)
        hosts.append(h)
        outs.append(torch.empty((n, n, n), device=dev, dtype=torch.float64))
        houts.append(torch.empty((n, n, n), dtype=torch.float64, pin_memory=True))
    stream = torch.cuda.current_stream(dev)
    steps = args.steps or 5

    def sweep(i):
        shape, r, _ = plan[i]
        mms.apply_f64(shape, r, coeffs[i], ins[i], outs[i])

    for _ in range(args.warmup):
        for i in range(len(plan)):
            sweep(i)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    ev = [[] for _ in plan]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        for i in range(len(plan)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sweep(i)
            b.record(stream)
            ev[i].append((a, b))
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed = max_over_ranks(t0.elapsed_time(t1) / 1e3, dist, dev)
    pts_step = sum(n ** 3 for _, _, n in plan)
    value = job_rate(world, pts_step * steps, elapsed)
    kms = [statistics.mean(a.elapsed_time(b) for a, b in e) for e in ev]
    # end to end: pinned host grids in, the FP64 sweeps, results out
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = 2
    e0.record(stream)
    for _ in range(e2e_steps):
        for i in range(len(plan)):
            ins[i].copy_(hosts[i], non_blocking=True)
            sweep(i)
            houts[i].copy_(outs[i], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
    # FP64 pipe: 2 FMAs per clock per SM (GB300's nominal 1.25 TFLOP/s FP64)
    fp64_peak = n_sm * 2 * 2 * sm_max_mhz * 1e6 / 1e12
    fmas = {"star": lambda r: 6 * r + 1, "box": lambda r: (2 * r + 1) ** 3}
    di = max(range(len(plan)), key=lambda i: kms[i])
    shape, r, n = plan[di]
    flops = 2 * fmas[shape](r) * n ** 3
    roof = {"bound": "alu", "achieved": flops / (kms[di] / 1e3) / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": flops / (kms[di] / 1e3) / 1e12 / fp64_peak, "traffic": captured_traffic(f"f64 {shape} r={r}", n ** 3),
            "kernel": f"f64_kernel {shape} r={r} {n}^3", "ms": kms[di],
            "peak_note": f"{n_sm} SMs x 2 FP64 FMA/clock x 2 flop x {sm_max_mhz:.0f} MHz (GB300's nominal FP64 rate)",
            "flop_per_point": 2 * fmas[shape](r)}
    sweeps = {f"{sh} r={rr}": {"ms": kms[i], "gpts": n_ ** 3 / (kms[i] / 1e3) / 1e9,
                                "fp64_tflops": 2 * fmas[sh](rr) * n_ ** 3 / (kms[i] / 1e3) / 1e12}
              for i, (sh, rr, n_) in enumerate(plan)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(lambda p, salt=0: oracle_sample(p, salt, plan), "GPoints/s",
                           "FP64 oracle, " + ", ".join(f"{sh} r={rr}" for sh, rr, _ in plan) +
                           ", on a seeded slab of {planes} output planes of each grid")
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GPoints/s", "n_gpus": world, "steps": steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD_NAMES[args.workload], "l2": "inputs larger than L2"},
                "roofline": roof, "sweeps": sweeps, "cpu_baseline": cpu,
                "e2e": {"value": job_rate(world, pts_step * e2e_steps, e2e_s), "unit": "GPoints/s",
                        "h2d_bytes_per_step": sum(h.numel() * 8 for h in hosts),
                        "d2h_bytes_per_step": sum(h.numel() * 8 for h in houts)},
                "gpu_launches": steps * len(plan), "clocks": clk,
                "peaks": {"hbm_gbs": hbm_peak, "source": peak_src}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _time(fn, reps=5):
    import torch
    fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def extras(mms, torch, dev, hbm_peak, alu_peak):
    """Timings outside the timed region, each with its error against the
    oracle: every sweep path on the box workload, the 1024^3 star r=4 on the
    CUDA cores and on the tensor cores, and brief runs of the wave, gradient,
    VTI and TTI workloads against the HBM roofline of their byte models."""
    out = {}
    for r in RADII:
        c = workloads.normal_coeffs("box", r, workload=2, salt=r)
        g = torch.Generator(device=dev).manual_seed(1000 + r)
        inp = mms.padded_empty(N, N, N, r, device=dev, zero=False)
        inp.uniform_(-1, 1, generator=g)
        host = inp.cpu().numpy()
        o = torch.empty((N, N, N), device=dev)
        for path in ("cuda_core", "naive", "tf32", "3xtf32", "bf16x3"):
            if mms.num_variants("box", r, path) == 0:
                continue
            ms = _time(lambda: mms.apply("box", r, c, inp, o, path=path))
            out[f"box_r{r}_{path}"] = {"ms": ms, "gpts": N ** 3 / ms / 1e6,
                                       "max_rel_err": sweep_error("box", r, c, host, o, salt=r)}
        del inp, o, host
    n = 1024
    inp = mms.padded_empty(n, n, n, 4, device=dev, zero=False)
    inp.uniform_(-1, 1, generator=torch.Generator(device=dev).manual_seed(7))
    host = inp.cpu().numpy()
    o = torch.empty((n, n, n), device=dev)
    c = workloads.fd8_star_coeffs()
    bytes_alg = 4 * ((n + 8) ** 3 + n ** 3)
    for path in ("cuda_core", "bf16x3"):
        ms = _time(lambda: mms.apply("star", 4, c, inp, o, path=path))
        out[f"star_r4_1024_{path}"] = {"ms": ms, "gpts": n ** 3 / ms / 1e6, "hbm_gbs": bytes_alg / ms / 1e6,
                                       "hbm_frac": bytes_alg / ms / 1e6 / hbm_peak,
                                       "variant": mms.default_variant("star", 4, path, n, n, n),
                                       "max_rel_err": sweep_error("star", 4, c, host, o, salt=4)}
    del inp, o, host
    torch.cuda.empty_cache()
    for name, fn in (("rtm512", extra_rtm), ("grad256", extra_grad), ("vti512", extra_vti),
                     ("tti512", extra_tti)):
        out[name] = fn(mms, torch, dev, hbm_peak)
        torch.cuda.empty_cache()
    return out


def _fill_interior(fields, r, gen):
    """Seeded U[-1, 1] in the interior of (nshots, Z, Y, X) fields, zero halo."""
    for f in fields:
        f.zero_()
        f[:, r:-r, r:-r, r:-r].uniform_(-1, 1, generator=gen)


def _roof_entry(ms_step, pts, bpp, hbm_peak, err, config):
    return {"ms_per_step": ms_step, "gpt_steps": pts / ms_step / 1e6, "bytes_per_point_step": bpp,
            "hbm_gbs": bpp * pts / ms_step / 1e6, "hbm_frac": bpp * pts / ms_step / 1e6 / hbm_peak,
            "max_rel_err": err, "config": config}


def extra_rtm(mms, torch, dev, hbm_peak, steps=20):
    """The acoustic forward workload in brief: 8 shots x 512^3, `steps`
    graph-launched steps (read a^n, a^{n-1}; write a^{n+1}: 16 B per
    point-step with m shared by the shots), from seeded random states; then
    one more step, checked at sampled points of shot 0."""
    import oracle
    from paper_2507_11067_gb300.wave import WavePropagator
    n, ns, R = 512, 8, 4
    w = workloads.WaveInputs(n, n, n, nshots=ns, nsteps=steps + 1, workload=4, noise=False)
    prop = WavePropagator(n, n, n, w.src, w.zrec, w.h, w.dt, sponge_width=w.sponge, sponge_a=w.sponge_a,
                          device=dev)
    prop.set_velocity(torch.from_numpy(w.v).to(dev))
    _fill_interior(prop.p, R, torch.Generator(device=dev).manual_seed(40))
    amps = torch.from_numpy(w.amp).to(dev).contiguous()
    rec = torch.empty((steps, ns, n, n), device=dev)
    ms = _time(lambda: mms.wave_forward(prop.desc, prop.coeffs, prop.m, amps[:steps], steps, prop.p[0],
                                        prop.p[1], rec, graph=True), reps=2) / steps
    # 3 runs of an even step count: p[1] holds a^n, p[0] a^{n-1}
    nxt = prop.new_fields(zero=True)
    mms.wave_step_to(prop.desc, prop.coeffs, prop.m, prop.p[1], prop.p[0], nxt, amps[steps])
    cur, prev = prop.p[1][0].cpu().numpy(), prop.p[0][0].cpu().numpy()
    src = w.src[0]
    pts = np.vstack([workloads.sample_points(n, n, n, 2000, workload=9, salt=40), [src]]).astype(np.int64)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    m = at_points(pts, (n, n, n), oracle.model_m(w.v[z, y, x], w.dt, w.h))
    ref = oracle.wave_step_points(R, prop.coeffs, m, (w.sponge, w.sponge_a), src, float(w.amp[steps, 0]),
                                  cur, prev, pts)
    idx = torch.from_numpy(pts).to(dev)
    got = nxt[0][idx[:, 2] + R, idx[:, 1] + R, idx[:, 0] + R].double().cpu().numpy()
    return _roof_entry(ms, ns * n ** 3, 16, hbm_peak, rel_err(got, ref),
                       f"{ns} shots x {n}^3, {steps} steps in one CUDA graph, from seeded random states")


def extra_grad(mms, torch, dev, hbm_peak):
    """The gradient workload (2 shots x 256^3, 200 steps, checkpoint every
    20): one whole gradient through WaveFunction; its three step kernels
    timed alone on seeded random fields; one adjoint step with its gradient
    term checked at every point against the oracle."""
    import oracle
    from paper_2507_11067_gb300.wave import WaveFunction, WavePropagator
    n, ns, nsteps, every, R = 256, 2, 200, 20, 4
    wt = workloads.WaveInputs(n, n, n, nshots=ns, nsteps=nsteps, workload=5, noise=True)
    w0 = workloads.WaveInputs(n, n, n, nshots=ns, nsteps=nsteps, workload=5, noise=False)
    prop = WavePropagator(n, n, n, w0.src, w0.zrec, w0.h, wt.dt, sponge_width=w0.sponge, sponge_a=w0.sponge_a,
                          device=dev)
    amps = torch.from_numpy(wt.amp).to(dev)
    with torch.no_grad():
        obs = WaveFunction.apply(torch.from_numpy(wt.v).to(dev), prop, amps, nsteps, every)
    v0 = torch.from_numpy(w0.v).to(dev)

    def gradient():
        vv = v0.clone().requires_grad_(True)
        (0.5 * ((WaveFunction.apply(vv, prop, amps, nsteps, every) - obs) ** 2).sum()).backward()

    ms = _time(gradient, reps=2)
    pts = ns * n ** 3
    bpp = 56.0 + 16.0 / ns
    f = [prop.new_fields() for _ in range(5)]
    _fill_interior(f, R, torch.Generator(device=dev).manual_seed(50))
    resid = torch.randn((ns, n, n), device=dev, generator=torch.Generator(device=dev).manual_seed(51))
    grad = torch.zeros((n, n, n), device=dev, dtype=torch.float64)
    t_fwd = _time(lambda: mms.wave_step_to(prop.desc, prop.coeffs, prop.m, f[0], f[1], f[2], amps[0]), reps=20)
    t_rec = _time(lambda: mms.wave_step_lap(prop.desc, prop.coeffs, prop.m, f[0], f[1], f[2], f[3], amps[0]),
                  reps=20)
    # the adjoint step in the variable the gradient carries (mu = m G lam
    # where every m > 0), and in lam for comparison
    t_adj = _time(lambda: mms.wave_adjoint_scaled(prop.desc, prop.coeffs, prop.m, f[0], f[4], resid, f[3], grad),
                  reps=20)
    t_adj_lam = _time(lambda: mms.wave_adjoint_lap(prop.desc, prop.coeffs, prop.m, f[0], f[4], resid, f[3], grad),
                      reps=20)
    # accuracy: lam^n (and mu^n) and the gradient term of one adjoint step
    # from seeded lam^{n+1}, lam^{n+2}, a^n (L a^n from the recompute kernel)
    _fill_interior(f, R, torch.Generator(device=dev).manual_seed(52))
    mms.wave_step_lap(prop.desc, prop.coeffs, prop.m, f[2], f[1], f[0], f[3], amps[0])
    l1, l2, an = (t.cpu().numpy().astype(np.float64) for t in (f[4], f[1], f[2]))
    grad.zero_()
    mms.wave_adjoint_lap(prop.desc, prop.coeffs, prop.m, f[4], f[1], resid, f[3], grad)
    prob = oracle.WaveProblem(R, prop.coeffs, oracle.model_m(w0.v, wt.dt, w0.h), (w0.sponge, w0.sponge_a),
                              w0.src, wt.amp, w0.zrec)
    gref = np.zeros((n, n, n))
    rh = resid.cpu().numpy().astype(np.float64)
    errs = [rel_err(f[1][sh].cpu().numpy(), prob.adjoint_step(l1[sh], l2[sh], rh[sh], an[sh], gref))
            for sh in range(ns)]
    errs.append(rel_err(grad.cpu().numpy(), gref))
    # the same in mu = m G lam: mu^{n+1}, mu^{n+2} = m G lam of the fields above
    mg = np.zeros_like(prob.m)
    gg = prob.gz[:, None, None] * prob.gy[None, :, None] * prob.gx[None, None, :]
    mg[R:-R, R:-R, R:-R] = prob.m[R:-R, R:-R, R:-R] * gg
    mu = [prop.new_fields(), prop.new_fields()]
    for t, lam in zip(mu, (l1, l2)):
        t.copy_(torch.from_numpy((lam * mg[None]).astype(np.float32)))
    m1, m2 = (t.cpu().numpy().astype(np.float64) for t in mu)
    grad.zero_()
    mms.wave_adjoint_scaled(prop.desc, prop.coeffs, prop.m, mu[0], mu[1], resid, f[3], grad)
    mms.grad_divide_m(prop.desc, prop.m, grad)
    gref = np.zeros((n, n, n))
    inner = mg > 0
    for sh in range(ns):
        lam1 = np.divide(m1[sh], mg, out=np.zeros_like(mg), where=inner)
        lam2 = np.divide(m2[sh], mg, out=np.zeros_like(mg), where=inner)
        errs.append(rel_err(mu[1][sh].cpu().numpy(), mg * prob.adjoint_step(lam1, lam2, rh[sh], an[sh], gref)))
    errs.append(rel_err(grad.cpu().numpy(), gref))
    return {"ms_per_gradient": ms, "gpt_steps": pts * nsteps / ms / 1e6, "bytes_per_point_step": bpp,
            "hbm_gbs": bpp * pts * nsteps / ms / 1e6, "hbm_frac": bpp * pts * nsteps / ms / 1e6 / hbm_peak,
            "forward_step_us": 1e3 * t_fwd, "recompute_step_us": 1e3 * t_rec, "adjoint_step_us": 1e3 * t_adj,
            "adjoint_lam_step_us": 1e3 * t_adj_lam, "adjoint": prop.adjoint,
            "max_rel_err": max(errs),
            "config": f"{ns} shots x {n}^3, {nsteps} steps, checkpoint every {every}; byte model: forward 16, "
                      f"recompute 20, adjoint 20 B per shot-point-step + FP64 gradient 16 B per point-step"}


def _aniso_setup(mms, torch, dev, kind, n, ns, steps):
    tti = kind == "tti"
    r = 4
    a = workloads.AnisoInputs(n, n, n, ns, steps + 1, workload=7 if tti else 6, tti=tti, noise=False)
    f = [mms.padded_empty(n, n, n, r, device=dev, nshots=ns) for _ in range(6)]
    py, pz, ss = mms.field_geometry(f[0])
    desc, keep = mms.wave_desc(n, n, n, r, ns, py, pz, ss, a.wave.sponge, a.wave.sponge_a, a.zrec, a.src)
    return a, f, desc, keep


def extra_vti(mms, torch, dev, hbm_peak, steps=10):
    """The VTI workload in brief: 4 shots x 512^3, `steps` fused steps from
    seeded random states (32 B per point-step); one more step checked at
    sampled points of shot 0."""
    from oracle import aniso
    n, ns, r = 512, 4, 4
    a, f, desc, _keep = _aniso_setup(mms, torch, dev, "vti", n, ns, steps)
    mv, rho = mms.padded_empty(n, n, n, r, device=dev), mms.padded_empty(n, n, n, r, device=dev)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    mms.vti_model(desc, d(a.vp), d(a.eps), d(a.delta), mv, rho, a.dt, a.h)
    cf = workloads.fd8_star_coeffs()
    amps = torch.from_numpy(a.amp).to(dev).contiguous()
    _fill_interior(f[:4], r, torch.Generator(device=dev).manual_seed(60))

    def run():
        cur = f[:4]
        for i in range(steps):
            mms.vti_step(desc, cf, mv, rho, cur[0], cur[1], cur[2], cur[3], cur[2], cur[3], amps[i])
            cur = [cur[2], cur[3], cur[0], cur[1]]
    ms = _time(run, reps=2) / steps
    # an even step count: f[0], f[1] hold the newest state again
    mms.vti_step(desc, cf, mv, rho, f[0], f[1], f[2], f[3], f[4], f[5], amps[steps])
    host = [t[0].cpu().numpy() for t in f[:4]]
    src = a.src[0]
    pts = np.vstack([workloads.sample_points(n, n, n, 2000, workload=9, salt=60), [src]]).astype(np.int64)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    mh_p, mv_p = aniso.vti_medium(a.vp[z, y, x], a.eps[z, y, x], a.delta[z, y, x], a.dt, a.h)
    oh, ov = aniso.vti_step_points(r, cf, at_points(pts, (n, n, n), mh_p), at_points(pts, (n, n, n), mv_p),
                                   (a.wave.sponge, a.wave.sponge_a), src, float(a.amp[steps, 0]), *host, pts)
    idx = torch.from_numpy(pts).to(dev)
    got = [t[0][idx[:, 2] + r, idx[:, 1] + r, idx[:, 0] + r].double().cpu().numpy() for t in (f[4], f[5])]
    err = max(rel_err(got[0], oh), rel_err(got[1], ov))
    return _roof_entry(ms, ns * n ** 3, ANISO["vti512"]["bytes_per_point_step"], hbm_peak, err,
                       f"{ns} shots x {n}^3, {steps} steps from seeded random states")


def extra_tti(mms, torch, dev, hbm_peak, steps=10):
    """The TTI workload in brief: 2 shots x 512^3, `steps` steps (two launches
    each; 88 B per point-step) from seeded random states; one more step
    checked at sampled points of shot 0."""
    from oracle import aniso
    n, ns, r = 512, 2, 4
    a, f, desc, _keep = _aniso_setup(mms, torch, dev, "tti", n, ns, steps)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    med = torch.empty((8, n, n, n), device=dev)
    mms.tti_model(desc, d(a.vp), d(a.vs), d(a.eps), d(a.delta), d(a.alpha), d(a.theta), d(a.phi), med, a.dt, a.h)
    work = torch.empty((4, ns, n, n, n), device=dev)
    w2, w1 = workloads.fd8_rows()
    amps = torch.from_numpy(a.amp).to(dev).contiguous()
    _fill_interior(f[:4], r, torch.Generator(device=dev).manual_seed(70))

    def run():
        cur = f[:4]
        for i in range(steps):
            mms.tti_step(desc, w2, w1, med, cur[0], cur[1], cur[2], cur[3], cur[2], cur[3], work, amps[i])
            cur = [cur[2], cur[3], cur[0], cur[1]]
    ms = _time(run, reps=2) / steps
    mms.tti_step(desc, w2, w1, med, f[0], f[1], f[2], f[3], f[4], f[5], work, amps[steps])
    host = [t[0].cpu().numpy() for t in f[:4]]
    src = a.src[0]
    pts = np.vstack([workloads.sample_points(n, n, n, 1000, workload=9, salt=70), [src]]).astype(np.int64)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    sel = lambda q: q[z, y, x]
    med_p = aniso.tti_medium(sel(a.vp), sel(a.vs), sel(a.eps), sel(a.delta), sel(a.alpha), a.dt, a.h)
    tilt_p = aniso.tilt_axis(sel(a.theta), sel(a.phi))
    full = lambda vals: at_points(pts, (n, n, n), vals)
    op, oq = aniso.tti_step_points(r, [full(v) for v in med_p], [full(v) for v in tilt_p],
                                   (a.wave.sponge, a.wave.sponge_a), src, float(a.amp[steps, 0]), *host, pts,
                                   w2, w1)
    idx = torch.from_numpy(pts).to(dev)
    got = [t[0][idx[:, 2] + r, idx[:, 1] + r, idx[:, 0] + r].double().cpu().numpy() for t in (f[4], f[5])]
    err = max(rel_err(got[0], op), rel_err(got[1], oq))
    return _roof_entry(ms, ns * n ** 3, ANISO["tti512"]["bytes_per_point_step"], hbm_peak, err,
                       f"{ns} shots x {n}^3, {steps} steps from seeded random states")


if __name__ == "__main__":
    sys.exit(main())
