"""Failure detection on the GPU without a fault: a kernel's bounded wait on a
barrier phase that nothing completes runs out, the device error word
reports it through mms_check_device, and the context keeps working."""
import time

import numpy as np
import pytest

import oracle
import paper_2507_11067_gb300 as mms
from paper_2507_11067_gb300 import _lib
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    mms.build()
    mms.load()
    assert torch.cuda.is_available()


def test_bounded_wait_times_out_and_the_context_stays_usable():
    mms.check_device()                       # starts clean
    t0 = time.perf_counter()
    _lib.selftest_timeout(20000)             # 20 ms
    with pytest.raises(mms.MMSError, match="TIMEOUT"):
        mms.check_device()
    assert time.perf_counter() - t0 >= 0.02  # the wait did run to its limit
    mms.check_device()                       # reading the word cleared it
    # the same context still computes a sweep correctly
    r, n = 2, (40, 33, 21)
    grid = workloads.uniform_grid(*n, r, workload=2, salt=61)
    c = workloads.normal_coeffs("box", r, workload=2, salt=61)
    out = mms.apply("box", r, c, mms.to_padded_device(grid, r), path="cuda_core")
    torch.cuda.synchronize()
    mms.check_device()
    ref = oracle.stencil("box", r, c, grid)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()
