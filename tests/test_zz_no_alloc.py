"""The allocation-free entry point lbm_field_moments, through the C ABI.

It must agree with an exactly rounded FP64 host sum of the downloaded field
and with the diagnostics the step kernels accumulate (lbm_get_diagnostics:
phi mass and first moments of the same time level) on two calls in a row
(its fixed scratch is reused), for FP64 and FP32 fields, on a side stream
and on the current stream, and reject lattices with more planes than its
scratch holds and fields that are not device memory of the current device.  Kept in a file
of its own that is collected last, so that it also runs after every other
test in the same process.
"""
import ctypes
import math

import numpy as np
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


def _host_moments(field):
    """Exactly rounded FP64 sums (math.fsum) of the downloaded field:
    sum psi and sum psi (x + 1/2), (y + 1/2), (z + 1/2), cell-centred."""
    a = field.detach().cpu().numpy().astype(np.float64)
    nz, ny, nx = a.shape[-3:]
    a = a.reshape(nz, ny, nx)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    return tuple(math.fsum(v.ravel()) for v in (a, a * x, a * y, a * z))


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
    host = _host_moments(phi)
    for call in range(2):                             # the scratch is reused by the second call
        st, m = _call(phi, w.nx, w.ny, w.nz, d.stream)
        assert st == 0, call
        for got, exact, key in zip(m, host, ("mass", "mx", "my", "mz")):
            assert abs(got - ref[key]) <= tol * abs(ref[key]), (case, call, key, got, ref[key])
            # FP64 accumulation of N terms: relative error well below 1e-12 here
            assert abs(got - exact) <= 1e-12 * abs(exact), (case, call, key, got, exact)


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


def test_field_moments_wrapper_side_stream_then_current_stream():
    """Through the Python wrapper (3-D tensor): two calls on a side stream,
    then, after a synchronise, one on the current stream; all three equal the
    exact host sums.  A tensor with a leading dimension > 1 is refused."""
    import torch
    from paper_2401_03041_gb300 import lbm
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(11)
    fa = torch.rand((13, 17, 19), generator=g, dtype=torch.float64).to(dev)
    fb = torch.rand((7, 5, 33), generator=g, dtype=torch.float64).to(dev).float()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    ra = lbm.field_moments(fa, stream=side)
    rb = lbm.field_moments(fb, stream=side)
    torch.cuda.synchronize(dev)
    rc = lbm.field_moments(fa)
    for got, field in ((ra, fa), (rb, fb), (rc, fa)):
        for v, e in zip(got, _host_moments(field)):
            assert abs(v - e) <= 1e-12 * abs(e), (v, e)
    assert rc == ra
    with pytest.raises(ValueError):
        lbm.field_moments(torch.zeros((2, 3, 4, 5), dtype=torch.float64, device=dev))


def test_field_moments_rejects_host_memory():
    """A host pointer is refused with LBM_ERR_ARG before anything runs."""
    import torch
    from paper_2401_03041_gb300 import lbm
    host = np.ones(2 * 3 * 4)
    out = (ctypes.c_double * 4)()
    st = lbm.lib().lbm_field_moments(ctypes.c_void_p(host.ctypes.data), 0, 2, 3, 4,
                                     ctypes.c_void_p(torch.cuda.current_stream(0).cuda_stream), out)
    assert st == -1
    assert "device memory" in lbm.lib().lbm_last_error().decode()
