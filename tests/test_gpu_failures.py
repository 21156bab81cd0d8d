"""Failure detection on the GPU without a fault: a bounded wait that runs out
is reported as a status, sticks to its domain and leaves the CUDA context
usable; a non-finite state is reported by the FP64 diagnostics.  The failures
are made on the host (a test knob that makes a copy wait expect bytes that
never arrive; a NaN written into the state through the ABI)."""
import time

import numpy as np
import pytest

from harness import gpu_domain, ragged_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_03041_gb300 import build
    build.build()


@pytest.mark.parametrize("kernel", ["bulk", "skew"])
def test_copy_wait_timeout_is_reported_and_context_survives(monkeypatch, kernel):
    from paper_2401_03041_gb300 import lbm
    w = ragged_workload("D3Q7", 15, walls=True, precision="fp32", shape=(80, 24, 12))
    monkeypatch.setenv("LBM_TEST_STALL", "1")
    d = gpu_domain(w, kernel=kernel)
    monkeypatch.delenv("LBM_TEST_STALL")
    t0 = time.time()
    d.step(1)
    with pytest.raises(lbm.LBMError) as e:
        d.synchronize(60000)
    assert e.value.status == -6                      # LBM_ERR_TIMEOUT
    assert time.time() - t0 < 30                     # bounded: ~2 s per wait
    with pytest.raises(lbm.LBMError) as e2:          # sticky on that domain
        d.step(1)
    assert e2.value.status == -6
    d.close()
    # the context is still usable: a fresh domain runs normally
    d2 = gpu_domain(w, kernel=kernel)
    d2.step(3)
    g = d2.diagnostics()
    assert not g["nonfinite"] and g["level"] == 3


def test_nonfinite_state_is_reported():
    from paper_2401_03041_gb300 import lbm
    w = ragged_workload("D3Q7", 15, walls=True, precision="fp64")
    d = gpu_domain(w)
    h = d.get_pdfs("h")
    h[3, 5, 7, 9] = np.nan
    d.set_pdfs("h", h)
    with pytest.raises(lbm.LBMError) as e:
        d.step_diagnostics(1)
    assert e.value.status == -5                      # LBM_ERR_NONFINITE
