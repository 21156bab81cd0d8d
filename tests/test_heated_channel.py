"""Pins of the planar heated channel's steady state (Sec. 3.1, App. A),
used by the GPU validation run: the layer-by-layer conduction / Stokes
solution meets every wall, interface and stress condition, agrees with the
appendix's closed form (read as stated in heated_channel), and drives the
interface from hot to cold when sigma_T < 0."""
import math

import numpy as np
import pytest

import heated_channel as hc


def _paper_channel(k_a, a=128.0):
    return hc.Channel(a=a, b=a, omega=2 * math.pi / (2 * a), T_h=20.0, T_c=10.0, T_0=4.0,
                      k_a=k_a, k_b=0.2, mu_a=0.2, mu_b=0.2, sigma_T=-5e-4)


@pytest.mark.parametrize("k_a", [0.2, 0.04])
def test_layer_solution_equals_appendix_closed_form(k_a):
    ch = _paper_channel(k_a)
    T, u, v = hc.solve(ch)
    Tp, up, vp = hc.printed(ch)
    x = np.linspace(0, 256, 41)[:, None]
    y = np.linspace(-128, 128, 81)[None, :]
    assert np.abs(T(x, y) - Tp(x, y)).max() < 1e-12
    assert np.abs(u(x, y) - up(x, y)).max() < 1e-12 * np.abs(up(x, y)).max()
    assert np.abs(v(x, y) - vp(x, y)).max() < 1e-12 * np.abs(vp(x, y)).max()


@pytest.mark.parametrize("k_a,mu_a", [(0.2, 0.2), (0.04, 0.2), (0.04, 0.5)])
def test_layer_solution_conditions(k_a, mu_a):
    ch = _paper_channel(k_a)
    ch.mu_a = mu_a
    T, u, v = hc.solve(ch)
    a, b, w = ch.a, ch.b, ch.omega
    x = np.linspace(0, 256, 17)
    assert np.abs(T(x, -b) - (ch.T_h + ch.T_0 * np.cos(w * x))).max() < 1e-12
    assert np.abs(T(x, a) - ch.T_c).max() < 1e-12
    for yw in (a, -b):
        assert np.abs(u(x, yw)).max() < 1e-15 and np.abs(v(x, yw)).max() < 1e-15
    e = 1e-5
    # T and k dT/dy continuous, v = 0 and u continuous on the interface
    # (one-sided differences over e on each side: O(e) residues)
    assert np.abs(T(x, e) - T(x, -e)).max() < 1e-5
    flux_a = ch.k_a * (T(x, 2 * e) - T(x, e)) / e
    flux_b = ch.k_b * (T(x, -e) - T(x, -2 * e)) / e
    assert np.abs(flux_a - flux_b).max() < 1e-4 * np.abs(flux_b).max()
    assert np.abs(v(x, e)).max() < 1e-9 and np.abs(u(x, e) - u(x, -e)).max() < 1e-9
    # tangential stress balance mu_a u_a' - mu_b u_b' = -sigma_T dT/dx on y = 0
    h = 1e-4
    dua = (u(x, 2 * h) - u(x, h)) / h
    dub = (u(x, -h) - u(x, -2 * h)) / h
    dTdx = (T(x + h, 0.0) - T(x - h, 0.0)) / (2 * h)
    lhs = ch.mu_a * dua - ch.mu_b * dub
    assert np.abs(lhs + ch.sigma_T * dTdx).max() < 1e-3 * np.abs(ch.sigma_T * dTdx).max()


def test_marangoni_flow_runs_from_hot_to_cold():
    """sigma_T < 0: surface tension is lowest above the hottest point (x = 0),
    so the interface flows away from it (u > 0 just right of x = 0) and the
    fluid rises towards the interface there (v > 0 below it at x = 0)."""
    T, u, v = hc.solve(_paper_channel(0.2))
    assert u(10.0, 1e-9) > 0 and u(-10.0, 1e-9) < 0
    assert v(0.0, -20.0) > 0
