"""Pins of the complex-step (forward-mode) derivatives of the oracle, the
exact reference for the adjoint's gradient."""
import dataclasses

import numpy as np

import workloads as W
from oracle import complex_step as cs
from oracle import model as om


def _tiny_capture():
    w = W.config5(n=16)
    return w.replace(nx=8, ny=8, nz=8,
                     patches=dataclasses.replace(w.patches, sx=2, sy=2, x0=[2, 4], y0=[2, 4],
                                                 intensity=[0.1, 0.1]),
                     droplets=[W.Droplet(4.3, 3.8, 3.6, 2.5)], target=(5.0, 4.0, 3.6))


def test_heat_gradient_is_exact_for_a_linear_quantity():
    """At rest in a periodic box, sum T grows by the patch's total source per
    step, so d(sum T)/dI_k = steps x (cells of patch k), exactly."""
    w = _tiny_capture()
    p = W.Params(**dict(w.params.__dict__, walls_z=False, sigma_T=0.0))
    w = w.replace(params=p, droplets=[])
    for k in range(2):
        assert abs(cs.heat_gradient(w, 5, k) - 5 * 4) < 1e-12


def test_capture_gradient_matches_central_differences():
    """The whole coupled step (moving droplet, Marangoni forcing, walls):
    complex-step dJ/dI_k equals central differences of the real oracle
    (h = 1e-2, O(h^2) truncation) to 1e-6, and J is the real run's J."""
    w = _tiny_capture()
    J, g = cs.capture_gradient(w, 6)

    def J_real(I):
        o = om.build(w.replace(patches=dataclasses.replace(w.patches, intensity=list(I))))
        o.step(6)
        return float(cs.capture_objective(o, w.target))

    I0 = np.array(w.patches.intensity)
    assert abs(J - J_real(I0)) < 1e-13 * J      # complex arithmetic rounds a little differently
    h = 1e-2
    fd = np.array([(J_real(I0 + h * e) - J_real(I0 - h * e)) / (2 * h) for e in np.eye(2)])
    assert np.abs(g - fd).max() < 1e-6 * np.abs(fd).max()
    assert np.abs(g).min() > 1e-8          # both patches move the droplet
