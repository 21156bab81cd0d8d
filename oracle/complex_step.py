"""Forward-mode derivatives of the oracle by complex-step differentiation.

Test infrastructure, like the rest of ``oracle/``: only the tests and the
scripts under tests/golden/ use it.

For a function F that is real-analytic in a real parameter s,
F(s + i h) = F(s) + i h F'(s) - h^2 F''(s) / 2 + ..., so
F'(s) = Im F(s + i h) / h + O(h^2) with no subtraction of nearby values
(Squire and Trapp, SIAM Review 40, 1998).  With h = 1e-30 the O(h^2) term is
far below FP64 rounding, so the result is the derivative to rounding: the
role a dual-number type plays in a compiled oracle.

The oracle's step is analytic in the heater intensities as long as every
operation on state-dependent values is: sums, products, quotients, sqrt of
|grad phi|^2 (never abs), and branches that depend only on positions.
``OracleLBM`` keeps to that, and allocates its outputs with the dtype of
its inputs, so a complex state propagates through a whole run.
"""
import numpy as np

from . import model

H = 1e-30


def _patch_mask(o, patches, k):
    return ((o.Zi == patches.z)
            & (o.Xi >= patches.x0[k]) & (o.Xi < patches.x0[k] + patches.sx)
            & (o.Yi >= patches.y0[k]) & (o.Yi < patches.y0[k] + patches.sy))


def _complex_run(workload, steps, k):
    """The oracle run of ``workload`` with heater intensity k perturbed by i H."""
    o = model.build(workload)
    o.h = o.h.astype(np.complex128)
    o.g = o.g.astype(np.complex128)
    if o.lb_thermal:
        o.f = o.f.astype(np.complex128)
    else:
        o.T = o.T.astype(np.complex128)
    o.q = o.q + 1j * H * _patch_mask(o, workload.patches, k)
    o.step(steps)
    return o


def capture_objective(o, target):
    """J = |sum(phi x) / sum(phi) - target|^2 of the current level, in the
    oracle's own dtype (the droplet-capture objective of the adjoint
    workload; a squared distance, not an absolute value, so it stays
    analytic)."""
    phi = o.macro()["phi"]
    m = phi.sum()
    c = [(phi * o.X).sum() / m, (phi * o.Y).sum() / m, (phi * o.Z).sum() / m]
    return sum((c[a] - target[a]) ** 2 for a in range(3))


def capture_gradient(workload, steps, patches=None):
    """J and dJ/dI_k after ``steps`` steps for the heater patches of
    ``workload`` (all of them, or the indices in ``patches``): one complex
    oracle run per patch."""
    idx = range(len(workload.patches.intensity)) if patches is None else patches
    J = None
    grad = []
    for k in idx:
        Jc = capture_objective(_complex_run(workload, steps, k), workload.target)
        J = Jc.real
        grad.append(Jc.imag / H)
    return float(J), np.array(grad)


def heat_gradient(workload, steps, k):
    """d(sum T)/dI_k after ``steps`` steps (used to pin the method: at rest
    in a periodic box it is steps times the patch's cell count)."""
    o = _complex_run(workload, steps, k)
    return float(o.macro()["T"].sum().imag / H)
