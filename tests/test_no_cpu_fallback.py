"""No CPU fallback anywhere in the product path: without a CUDA device the
benchmark's own arm, the smoke test and the binding stop with an error
instead of computing anything on the host (the oracle runs only in tests,
smoke's checks and the benchmark's reference and CPU-baseline legs)."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_11067_gb300 as mms  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")


@pytest.mark.parametrize("workload", ["box512", "rtm512", "vti512", "fp64_512"])
def test_benchmark_arm_fails_without_a_gpu(workload):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", workload, "--steps", "1",
                        "--warmup", "3", "--no-cpu-baseline"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode != 0
    assert not any(l.startswith("{") for l in r.stdout.splitlines())


def test_smoke_fails_without_a_gpu():
    import __graft_entry__
    with pytest.raises((AssertionError, RuntimeError)):
        __graft_entry__.smoke()


def test_binding_never_computes_on_host_tensors():
    inp = mms.padded_empty(8, 8, 8, 1, device="cpu")
    out = torch.full((8, 8, 8), 7.0)
    with pytest.raises(mms.MMSError):
        mms.apply("star", 1, np.ones(9), inp, out)
    assert torch.all(out == 7.0)
