"""Checkpoint / resume through the C ABI (lbm_save_state / lbm_load_state):
a run resumed from a saved state continues bit for bit as the run that was
never interrupted, in the same domain or in a fresh one; a state of another
kind of domain is rejected."""
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


def _fields(d):
    return {k: v.detach().cpu().numpy() for k, v in d.fields(dtype="f64").items()}


@pytest.mark.parametrize("thermal,precision,shape", [("D3Q7", "fp32", (80, 24, 12)),
                                                     ("RK4", "fp64", (40, 20, 13))])
def test_resume_is_bitwise(thermal, precision, shape):
    w = ragged_workload(thermal, 15, walls=True, precision=precision, shape=shape)
    d = gpu_domain(w)
    d.step(5)
    state = d.save_state()
    d.step(7)
    ref = _fields(d)
    assert d.level() == 12
    d.load_state(state)
    assert d.level() == 5
    d.step(7)
    again = _fields(d)
    fresh = gpu_domain(w)
    fresh.load_state(state)
    fresh.step(7)
    other = _fields(fresh)
    for k in ref:
        assert np.array_equal(ref[k], again[k]), k
        assert np.array_equal(ref[k], other[k]), k


def test_state_of_another_domain_is_rejected():
    from paper_2401_03041_gb300 import lbm
    a = gpu_domain(ragged_workload("D3Q7", 15, walls=True, precision="fp64", shape=(40, 20, 13)))
    b = gpu_domain(ragged_workload("D3Q7", 15, walls=True, precision="fp64", shape=(40, 20, 14)))
    with pytest.raises(lbm.LBMError) as e:
        b.load_state(a.save_state())
    assert e.value.status == -1
    with pytest.raises(lbm.LBMError) as e:
        a.load_state(b"not a state" * 10)
    assert e.value.status == -1
