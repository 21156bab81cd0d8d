"""The allocation-free entry point lbm_field_moments, through the C ABI.

It must agree with the diagnostics the step kernels accumulate
(lbm_get_diagnostics: phi mass and first moments of the same time level) on
two calls in a row (its fixed scratch is reused), for FP64 and FP32 fields,
and reject lattices with more planes than its scratch holds.  Kept in a file
of its own that is collected last, so that it also runs after every other
test in the same process.
"""
import ctypes

import pytest

import workloads as W
from harness import gpu_domain, ragged_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_03041_gb300 import build
    build.build()


def _call(field, nx, ny, nz, stream):
    """lbm_field_moments straight through ctypes; returns (status, 4 sums)."""
    import torch
    from paper_2401_03041_gb300 import lbm
    out = (ctypes.c_double * 4)()
    st = lbm.lib().lbm_field_moments(ctypes.c_void_p(field.data_ptr()),
                                     0 if field.dtype == torch.float64 else 1,
                                     nx, ny, nz, ctypes.c_void_p(stream.cuda_stream), out)
    return st, tuple(out)


@pytest.mark.parametrize("case", ["fp64_droplet_32cube", "fp32_ragged_walls"])
def test_field_moments_match_step_diagnostics(case):
    if case == "fp64_droplet_32cube":
        w, dtype, tol = W.config1(), "f64", 1e-12
    else:
        w, dtype, tol = ragged_workload("D3Q7", 15, walls=True, precision="fp32",
                                        shape=(80, 24, 12)), "f32", 1e-10
    d = gpu_domain(w)
    d.step(7)
    ref = d.diagnostics()
    phi = d.fields(1, dtype=dtype)["phi"]           # device tensor [nz][ny][nx], same level
    assert phi.is_contiguous()
    for call in range(2):                             # the scratch is reused by the second call
        st, m = _call(phi, w.nx, w.ny, w.nz, d.stream)
        assert st == 0, call
        for got, key in zip(m, ("mass", "mx", "my", "mz")):
            assert abs(got - ref[key]) <= tol * abs(ref[key]), (case, call, key, got, ref[key])


def test_field_moments_rejects_more_planes_than_scratch():
    import torch
    from paper_2401_03041_gb300 import lbm
    dev = torch.device("cuda", 0)
    field = torch.zeros(8, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    # nz one beyond the limit: rejected before anything is launched or read
    st, _ = _call(field, 1, 1, 4097, stream)
    assert st == -1
    assert "LBM_MOMENTS_MAX_PLANES" in lbm.lib().lbm_last_error().decode()
    # the library still works afterwards
    st, m = _call(field, 2, 2, 2, stream)
    assert st == 0 and m == (0.0, 0.0, 0.0, 0.0)
