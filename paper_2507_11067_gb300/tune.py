"""Tile autotuner of the sweep kernels.

For one (shape, radius, path) and grid size, every tile variant the library
offers (mms_num_variants) is timed with CUDA events on the current stream;
the fastest is registered with mms_set_variant (so MMS_PATH_AUTO and
variant -1 use it) and recorded in a JSON table keyed by GPU name, shape,
radius, path and grid size.  The committed table ``tuned.json`` is loaded by
``load_table()``; the paper picks a tile size per kernel by hand (Table I),
this picks it by measurement.
"""
from __future__ import annotations

import json
import os

from . import _lib

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def _key(gpu, shape, r, path, n):
    return f"{gpu}|{shape}|r{r}|{path}|{n[0]}x{n[1]}x{n[2]}"


def time_variants(shape, r, path, inp, out, coeffs, reps=10, warmup=3):
    """ms per sweep of every variant (list indexed by variant)."""
    import torch
    res = []
    for v in range(_lib.num_variants(shape, r, path)):
        for _ in range(warmup):
            _lib.apply(shape, r, coeffs, inp, out, path=path, variant=v)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            _lib.apply(shape, r, coeffs, inp, out, path=path, variant=v)
        e.record()
        torch.cuda.synchronize()
        res.append(s.elapsed_time(e) / reps)
    return res


def tune(shape, r, path, nx, ny, nz, coeffs=None, reps=10, table=TABLE, write=True, seed=0):
    """Time all variants on a seeded U[-1,1] grid, register and record the best."""
    import torch
    import numpy as np
    dev = torch.cuda.current_device()
    alloc = _lib.padded_empty2d if _lib.SHAPES[shape] in _lib.PLANAR else _lib.padded_empty
    inp = alloc(nx, ny, nz, r, device=dev, zero=False)
    inp.uniform_(-1, 1, generator=torch.Generator(device=dev).manual_seed(seed))
    out = torch.empty((nz, ny, nx), device=dev)
    if coeffs is None:
        n = _lib.n_coeffs(shape, r)
        coeffs = np.random.default_rng(seed).normal(0, n ** -0.5, n).astype(np.float32)
    ms = time_variants(shape, r, path, inp, out, coeffs, reps=reps)
    best = int(min(range(len(ms)), key=lambda i: ms[i]))
    _lib.set_variant(shape, r, path, best)
    if write:
        gpu = torch.cuda.get_device_name(dev)
        data = json.load(open(table)) if os.path.exists(table) else {}
        data[_key(gpu, shape, r, path, (nx, ny, nz))] = {"variant": best, "ms": ms}
        with open(table, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    return best, ms


def tune_auto(shape, r, nx, ny, nz, reps=10, table=TABLE, seed=0):
    """Tune the CUDA-core path and, where built, the BF16x3 tensor-core path
    (FP32-level accuracy) for (shape, r); the tensor-core variant is recorded
    (and so chosen by MMS_PATH_AUTO) only if it is faster."""
    import torch
    best_cc, ms_cc = tune(shape, r, "cuda_core", nx, ny, nz, reps=reps, table=table, seed=seed)
    out = {"cuda_core": (best_cc, ms_cc)}
    if _lib.num_variants(shape, r, "bf16x3"):
        best_tc, ms_tc = tune(shape, r, "bf16x3", nx, ny, nz, reps=reps, table=table, write=False,
                              seed=seed)
        out["bf16x3"] = (best_tc, ms_tc)
        gpu = torch.cuda.get_device_name(torch.cuda.current_device())
        data = json.load(open(table)) if os.path.exists(table) else {}
        key = _key(gpu, shape, r, "bf16x3", (nx, ny, nz))
        if min(ms_tc) < min(ms_cc):
            data[key] = {"variant": best_tc, "ms": ms_tc, "beats_cuda_core_ms": min(ms_cc)}
        else:
            data.pop(key, None)
            _lib.set_variant(shape, r, "bf16x3", -1)
        with open(table, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    return out


def load_table(table=TABLE, n=None):
    """Register the recorded best variants for this GPU (largest grid wins
    when several sizes were tuned, unless n = (nx, ny, nz) picks one);
    returns {(shape, r, path): variant} of what it registered."""
    import torch
    if not os.path.exists(table):
        return {}
    gpu = torch.cuda.get_device_name(torch.cuda.current_device())
    data = json.load(open(table))
    chosen = {}
    for k, v in data.items():
        g, shape, rr, path, size = k.split("|")
        if g != gpu:
            continue
        dims = tuple(int(s) for s in size.split("x"))
        if n is not None and dims != tuple(n):
            continue
        key = (shape, int(rr[1:]), path)
        vol = dims[0] * dims[1] * dims[2]
        if key not in chosen or vol > chosen[key][0]:
            chosen[key] = (vol, v["variant"])
    registered = {}
    for (shape, r, path), (_, var) in chosen.items():
        # a table written by a build with more variants than this one is skipped
        if var < _lib.num_variants(shape, r, path):
            _lib.set_variant(shape, r, path, var)
            registered[(shape, r, path)] = var
    return registered


# The grids the committed table is tuned on: the 3D kernels at the sizes the
# benchmark times (box 512^3, star 1024^3), Table I's 2D kernels on one
# 8192^2 plane.
STANDARD = [(shape, r, n) for r in (1, 2, 3, 4)
            for shape, n in (("box", (512, 512, 512)), ("star", (1024, 1024, 1024)),
                             ("star2d", (8192, 8192, 1)), ("box2d", (8192, 8192, 1)))]


def retune(table=TABLE, reps=10):
    """Re-measure every (shape, radius) of STANDARD on this GPU (CUDA-core
    variants, and the BF16x3 tensor-core variants kept where faster) and
    rewrite their rows of `table`; returns {(shape, r): results}."""
    out = {}
    for shape, r, n in STANDARD:
        out[(shape, r)] = tune_auto(shape, r, *n, reps=reps, table=table)
        best = {p: min(ms) for p, (_, ms) in out[(shape, r)].items()}
        print(f"{shape} r={r} {n[0]}x{n[1]}x{n[2]}: " + ", ".join(f"{p} {v:.3f} ms" for p, v in best.items()),
              flush=True)
    return out


if __name__ == "__main__":
    import sys
    from . import build
    build()
    _lib.load()
    retune(table=sys.argv[1] if len(sys.argv) > 1 else TABLE)
