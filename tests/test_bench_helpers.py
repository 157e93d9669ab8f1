"""bench.py's bookkeeping on CPU: the traffic of a committed ncu capture is
used only while the kernel's code is the one captured (a comment-insensitive
hash), the roofline helpers count what they say, and the reference arm (the
oracle on the host cores) prints the contract's JSON line on rank 0 only."""
import json
import os

import pytest

import bench


def test_code_hash_ignores_comments_but_not_code(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text("// header\n__global__ void k(float *x)\n{\n    x[0] = 1.f;  // one\n}\n")
    h = bench.code_hash(str(a))
    a.write_text("/* another\n   header */\n__global__ void k(float *x)\n{\n\n    x[0] = 1.f;\n}\n")
    assert bench.code_hash(str(a)) == h
    a.write_text("__global__ void k(float *x)\n{\n    x[0] = 2.f;\n}\n")
    assert bench.code_hash(str(a)) != h


def test_committed_traffic_matches_the_committed_sources():
    # every recorded capture names sources that exist, and the keys the bench
    # looks up for its default and wave workloads resolve
    t = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for key, rec in t.items():
        assert os.path.exists(os.path.join(bench.ROOT, rec["capture"])), key
        for f in rec["sources"]:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2507_11067_gb300", "csrc", f)), (key, f)
    assert bench.captured_traffic("bf16x3 box r=2 v0", 512 ** 3) == pytest.approx(
        t["bf16x3 box r=2 v0"]["dram_bytes_per_point"] * 512 ** 3)
    assert bench.captured_traffic("no such kernel", 10) is None


def test_traffic_goes_null_when_a_source_changes(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_2507_11067_gb300" / "csrc").mkdir(parents=True)
    src = root / "paper_2507_11067_gb300" / "csrc" / "k.cu"
    src.write_text("__global__ void k() {}\n")
    rec = {"k r=1": {"dram_bytes_per_point": 8.0, "capture": "profiles/k.md", "size": "1",
                     "sources": {"k.cu": bench.code_hash(str(src))}}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.captured_traffic("k r=1", 100) == 800.0
    src.write_text("// same kernel, new comment\n__global__ void k() {}\n")
    assert bench.captured_traffic("k r=1", 100) == 800.0
    src.write_text("__global__ void k() { int a = 0; }\n")
    assert bench.captured_traffic("k r=1", 100) is None


def test_tensor_core_dense_work_per_point():
    # per output plane a tile (4 subtiles of TXO = 16 - 2r rounded down to a
    # multiple of 4 outputs, TY = 32 - 2r rows) runs 128 x N x 16 MMAs,
    # N = (2r+1) TXO rounded up to 16, for each plane reached in z, times 3
    # split products (BF16x3)
    assert bench.tc_dense_flop_per_pt("bf16x3", 2) == pytest.approx(2 * 128 * 64 * 16 * 5 * 3 / (4 * 12 * 28))
    assert bench.tc_dense_flop_per_pt("bf16x3", 4) == pytest.approx(2 * 128 * 80 * 16 * 9 * 3 / (4 * 8 * 24))
    assert bench.tc_dense_flop_per_pt("tf32", 1) == pytest.approx(2 * 128 * 48 * 16 * 3 / (4 * 12 * 30))
    assert bench.tc_dense_flop_per_pt("bf16x3", 3) == pytest.approx(2 * 128 * 64 * 16 * 7 * 3 / (4 * 8 * 26))
    assert bench.tc_dense_flop_per_pt("bf16x3", 4, planar=True) == pytest.approx(2 * 128 * 80 * 16 * 3 / (4 * 8 * 24))


def test_tensor_core_roofline_is_the_stencils_own_floor():
    # box r=2 512^3 in 0.4734 ms: the binding floor is HBM (4 (516^3 + 512^3)
    # bytes at 6690.8 GB/s = 0.162 ms, far above 250 flop/pt at the BF16
    # peak), so frac = algorithmic bytes / time / measured HBM, and the dense
    # MMA work goes to the side fields
    n, sec = 512 ** 3, 0.4734e-3
    b = 4.0 * (516 ** 3 + 512 ** 3)
    r = bench.tc_roofline("box", 2, "bf16x3", n, b, sec, 6690.8, 1714.1, "measured sustained")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6690.8
    assert r["frac"] == pytest.approx(b / sec / 1e9 / 6690.8)
    assert r["frac"] == pytest.approx(0.343, abs=1e-3)
    dense = bench.tc_dense_flop_per_pt("bf16x3", 2) * n
    assert r["dense_tflops"] == pytest.approx(dense / sec / 1e12)
    assert r["tensor_pipe_frac"] == pytest.approx(dense / sec / 1e12 / 1714.1)
    # a hypothetical sweep whose useful flops outrun the tensor floor reports
    # against the tensor peak (TF32 at 1.1/2.25 of BF16)
    r = bench.tc_roofline("box", 4, "tf32", n, 1.0, 1e-3, 6690.8, 1714.1, "x")
    assert r["bound"] == "tensor" and r["peak"] == pytest.approx(1714.1 * 1.1 / 2.25)
    assert r["frac"] == pytest.approx(2 * 729 * n / 1e-3 / 1e12 / (1714.1 * 1.1 / 2.25))


def test_job_rate_and_fp32_peak():
    assert bench.job_rate(4, 1e9, 2.0) == pytest.approx(2.0)
    assert bench.fp32_alu_peak_tflops(152, 2070.0) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


@pytest.mark.parametrize("workload", ["box512", "rtm512", "vti512"])
def test_reference_arm_prints_the_contract_line(workload):
    # the oracle on the host cores, on tiny samples (MMS_REF_STEP_SECONDS)
    import json
    import subprocess
    import sys
    env = dict(os.environ, MMS_REF_STEP_SECONDS="0.05", OMP_NUM_THREADS="2")
    cmd = [sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--workload", workload,
           "--steps", "2", "--warmup", "3"]
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    assert d["cpu_baseline"]["value"] == d["value"] == d["e2e"]["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] and "model" not in d["config"]
    # other ranks of a torchrun launch exit quietly
    out = subprocess.run(cmd, env=dict(env, RANK="1", WORLD_SIZE="2"), capture_output=True, text=True,
                         timeout=120, cwd=bench.ROOT)
    assert out.returncode == 0 and not out.stdout.strip()


def test_sweep_error_is_the_max_relative_error_at_the_sample_points():
    # an output equal to the oracle's sweep has error 0; one off by a known
    # amount at one sampled point reports that amount over max |oracle|
    import numpy as np
    import oracle
    import workloads
    r, n = 2, (21, 17, 13)
    grid = workloads.uniform_grid(*n, r, workload=2, salt=5)
    c = workloads.normal_coeffs("box", r, workload=2, salt=5)
    exact = oracle.stencil("box", r, c, grid)
    assert bench.sweep_error("box", r, c, grid, exact) == 0.0
    pts = workloads.sample_points(n[0], n[1], n[2], 2000, workload=9, salt=0)
    bad = exact.copy()
    x, y, z = pts[0]
    bad[z, y, x] += 1e-3
    ref = oracle.stencil_points("box", r, c, grid, pts)
    assert bench.sweep_error("box", r, c, grid, bad) == pytest.approx(1e-3 / np.abs(ref).max())
    # the planar form
    g2 = workloads.uniform_grid2d(40, 30, 1, 3, workload=6, salt=1)
    c2 = workloads.normal_coeffs("box2d", 3, workload=6, salt=1)
    assert bench.sweep_error("box2d", 3, c2, g2, oracle.stencil2d("box2d", 3, c2, g2)) == 0.0


def test_at_points_places_values_only_at_the_points():
    import numpy as np
    pts = np.array([[1, 2, 3], [0, 0, 0]])
    a = bench.at_points(pts, (4, 5, 6), [7.0, 8.0])
    assert a.shape == (4, 5, 6) and a[3, 2, 1] == 7.0 and a[0, 0, 0] == 8.0 and a.sum() == 15.0


def test_cpu_baseline_times_all_cores_and_one_core():
    import oracle
    calls = []

    def sample(planes, salt=0):
        calls.append(oracle.set_threads(0))
        return bench.oracle_sample(planes, salt, [("box", 1, 24)])

    before = oracle.set_threads(0)
    out = bench.cpu_baseline(sample, "GPoints/s", "slab of {planes} planes", budget_s=0.01)
    assert oracle.set_threads(0) == before               # the count is restored
    assert out["cores"] == before and out["one_core"]["cores"] == 1 and 1 in calls
    assert out["value"] > 0 and out["one_core"]["value"] > 0
    assert "{planes}" not in out["sample"] and "{planes}" not in out["one_core"]["sample"]
