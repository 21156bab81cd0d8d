"""Validation of the CUDA path on the planar heated channel (Sec. 3.1,
App. A; the paper's Tables 1 and 2 give its l2 errors after 4e5 steps at
512 x 256).

Here the same channel at a quarter of the paper's resolution: 128 x 64 cells
in x-z (two periods of the wall modulation, a = b = 32, so omega a = pi as in
the paper), 8 cells deep in the periodic y direction, FP64.  Parameters as in
the paper: nu = 0.2 in both fluids, M = 0.05, sigma_ref = 2.5e-2,
sigma_T = -5e-4, T_h = 20, T_c = 10, T_0 = 4, kappa_b = 0.2 (lower fluid,
phi = 0) and kappa_a = 0.2 or 0.04 (upper fluid, phi = 1), xi = 4; rho c_p = 1.
The run starts from the flat tanh interface, the conduction temperature and
rest, and is compared after 24000 and 30000 steps with the steady state of
tests/heated_channel.py (the errors must have settled) in the l2 norm of the
paper, for the LB and RK4 energy solvers.  The bounds allow for the coarser
grid (the interface is 4 cells wide in a 64-cell channel, against 256 in the
paper); the measured values are printed.
"""
import math

import numpy as np
import pytest

import heated_channel as hc

pytestmark = pytest.mark.gpu

NX, NY, NZ = 128, 8, 64


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_03041_gb300 import build
    build.build()


def _run(thermal, k_a, checkpoints):
    from paper_2401_03041_gb300 import lbm
    ch = hc.Channel(a=NZ / 2, b=NZ / 2, omega=2 * math.pi * 2 / NX, T_h=20.0, T_c=10.0, T_0=4.0,
                    k_a=k_a, k_b=0.2, mu_a=0.2, mu_b=0.2, sigma_T=-5e-4)
    T_ex, u_ex, v_ex = hc.solve(ch)
    d = lbm.Domain(NX, NY, NZ, "fp64", thermal, 15)
    d.set_params(nu_L=0.2, nu_H=0.2, mobility=0.05, xi=4.0, sigma_ref=2.5e-2, sigma_T=-5e-4,
                 T_ref=15.0, alpha_L=0.2, alpha_H=k_a, walls_z=True, T_bottom=20.0, T_top=10.0,
                 T_bottom_amp=4.0, T_bottom_waves=2)
    d.init_droplets([])
    Z, Y, X = np.meshgrid(np.arange(NZ) + 0.5, np.arange(NY) + 0.5, np.arange(NX) + 0.5, indexing="ij")
    yp = Z - NZ / 2
    phi = 0.5 + 0.5 * np.tanh(2.0 * yp / 4.0)
    c15, w15 = lbm.stencil(15)
    d.set_pdfs("h", np.array(w15)[:, None] * phi.ravel()[None, :])
    d.set_pdfs("g", np.zeros((27, phi.size)))
    T0 = T_ex(X, yp)
    if thermal.startswith("D3Q"):
        _, wf = lbm.stencil(int(thermal[3:]))
        d.set_pdfs("f", np.array(wf)[:, None] * T0.ravel()[None, :])
    else:
        d.set_pdfs("T", T0.ravel()[None, :])
    out = []
    done = 0
    for n in checkpoints:
        d.step(n - done)
        done = n
        f = {k: v.detach().cpu().numpy() for k, v in d.fields(dtype="f64").items()}
        T = f["T"][:, 0, :]
        ux, uz = f["u"][0][:, 0, :], f["u"][2][:, 0, :]
        x, y = X[:, 0, :], yp[:, 0, :]
        eT = hc.l2(T, T_ex(x, y))
        eu = hc.l2(np.hypot(ux, uz), np.hypot(u_ex(x, y), v_ex(x, y)))
        out.append((n, eT, eu, float(np.abs(f["u"][1]).max())))
    d.close()
    return out


@pytest.mark.parametrize("thermal", ["D3Q7", "RK4"])
@pytest.mark.parametrize("k_a", [0.2, 0.04])
def test_planar_heated_channel_steady_state(thermal, k_a):
    res = _run(thermal, k_a, (24000, 30000))
    print("heated channel", thermal, "k*", k_a / 0.2, [(n, f"{eT:.3e}", f"{eu:.3e}") for n, eT, eu, _ in res])
    (_, eT1, eu1, _), (_, eT2, eu2, uy) = res
    assert abs(eT2 - eT1) <= 0.05 * eT2 + 1e-6 and abs(eu2 - eu1) <= 0.05 * eu2   # settled
    assert eT2 < 1e-2
    assert eu2 < 0.3
    assert uy < 1e-12                                                              # stays 2D
