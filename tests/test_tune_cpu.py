"""The autotuner's table on CPU: which variants load_table registers for a
GPU, which grid wins when several sizes were tuned, and that AUTO follows
the registered tensor-core entries.  load_table's two torch.cuda queries
(the device and its name) are replaced here; registering a variant is
host-only, so the library's own choice (mms_default_variant, mms_auto_path)
is read back as it stands."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_11067_gb300 as mms  # noqa: E402
from paper_2507_11067_gb300 import tune  # noqa: E402

SHAPES = ("star", "box", "star2d", "box2d")
PATHS = ("cuda_core", "tf32", "3xtf32", "bf16x3")


@pytest.fixture
def gpu(monkeypatch):
    mms.build()
    mms.load()
    name = {"v": "NVIDIA GB300"}
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda d=None: name["v"])
    yield name
    for shape in SHAPES:
        for r in range(1, 5):
            for path in PATHS:
                if mms.num_variants(shape, r, path):
                    mms.set_variant(shape, r, path, -1)


def test_committed_table_registers_its_fastest_variants(gpu):
    data = json.load(open(tune.TABLE))
    chosen = tune.load_table()
    assert len(chosen) == len(data)           # one grid size per kernel in the committed table
    for k, v in data.items():
        g, shape, rr, path, size = k.split("|")
        r = int(rr[1:])
        assert g == gpu["v"]
        # the timings cover every variant of this build, and the recorded one is their fastest
        assert len(v["ms"]) == mms.num_variants(shape, r, path)
        assert v["variant"] == int(np.argmin(v["ms"]))
        assert chosen[(shape, r, path)] == v["variant"]
        assert mms.default_variant(shape, r, path) == v["variant"]
        if path == "bf16x3":                  # kept only where it beat the CUDA cores
            assert min(v["ms"]) < v["beats_cuda_core_ms"]
            cc = data[k.replace("bf16x3", "cuda_core")]
            assert v["beats_cuda_core_ms"] == pytest.approx(min(cc["ms"]))
    for r in (2, 3, 4):
        assert mms.auto_path("box", r) == "bf16x3"
    for shape, r in (("box", 1), ("star", 4), ("star2d", 2), ("box2d", 3)):
        assert mms.auto_path(shape, r) == "cuda_core"


def test_other_gpus_get_nothing(gpu):
    gpu["v"] = "some other GPU"
    assert tune.load_table() == {}
    assert mms.auto_path("box", 2) == "cuda_core"
    assert mms.default_variant("star", 4, "cuda_core") == 0


def test_largest_grid_wins_unless_a_size_is_named(gpu, tmp_path):
    t = tmp_path / "t.json"
    rec = {
        "NVIDIA GB300|star|r2|cuda_core|64x64x64": {"variant": 3, "ms": []},
        "NVIDIA GB300|star|r2|cuda_core|512x512x512": {"variant": 5, "ms": []},
        "NVIDIA GB300|star|r2|cuda_core|128x128x128": {"variant": 1, "ms": []},
        "NVIDIA GB300|star|r3|cuda_core|64x64x64": {"variant": 99, "ms": []},   # beyond this build
        "other|star|r1|cuda_core|64x64x64": {"variant": 2, "ms": []},
    }
    t.write_text(json.dumps(rec))
    assert tune.load_table(str(t)) == {("star", 2, "cuda_core"): 5}
    assert mms.default_variant("star", 2, "cuda_core") == 5
    assert mms.default_variant("star", 3, "cuda_core") == 0
    assert tune.load_table(str(t), n=(128, 128, 128)) == {("star", 2, "cuda_core"): 1}
    assert mms.default_variant("star", 2, "cuda_core") == 1
    assert tune.load_table(str(tmp_path / "missing.json")) == {}
