"""The discrete adjoint (lbm_adjoint_step / lbm_adjoint_run) through the C ABI.

Checks, all in FP64:
  * per step, exact adjoint: <lam, (Phi(s + e d) - Phi(s - e d)) / 2e> =
    <(dPhi/ds)^T lam, d> for random lam and d (walls and periodic, D3Q15 and
    D3Q27 phase field, unequal viscosities, gravity, background gradient,
    heat sources; every energy solver: thermal LB D3Q7/15/19/27, RK2, RK4);
  * the exact gradient dJ/dI of the droplet-capture objective against central
    finite differences of the FP64 *oracle* (independent of the CUDA path) on
    the 16^3 adjoint workload (40 steps; D3Q7, D3Q19, RK4, RK2), and against
    the oracle's exact complex-step derivatives (stored golden values);
  * on the full 64^3, 2000-step workload the exact linearisation diverges
    (the interface normal's derivative in far-field tails); the adjoint that
    holds the normal fixed where |4 phi (1 - phi) / xi| > 30 |grad phi| is
    checked there against central differences of the GPU forward;
  * checkpoint spacing does not change the result (bitwise);
  * the torch.autograd.Function wrapper returns the same gradient.
"""
import dataclasses

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


def _with_intensity(w, intensity):
    return w.replace(patches=dataclasses.replace(w.patches, intensity=list(intensity)))


def _third(d):
    """The energy solver's state: f (thermal LB) or the T field (RK)."""
    return "T" if d.thermal.startswith("RK") else "f"


def _state(d):
    return np.concatenate([d.get_pdfs("h").ravel(), d.get_pdfs("g").ravel(), d.get_pdfs(_third(d)).ravel()])


def _set_state(d, s, qh, N):
    nh, ng = qh * N, 27 * N
    d.set_pdfs("h", s[:nh].reshape(qh, -1))
    d.set_pdfs("g", s[nh:nh + ng].reshape(27, -1))
    third = _third(d)
    d.set_pdfs(third, s[nh + ng:].reshape(-1, N) if third == "f" else s[nh + ng:])


def _periodic_case(q_phase, thermal="D3Q7"):
    w = ragged_workload(thermal, q_phase, walls=False, precision="fp64", shape=(12, 10, 8))
    return w


@pytest.mark.parametrize("case", ["walls_patches_q15", "periodic_q15", "periodic_q27", "walls_patches_q15_f19",
                                  "periodic_q27_f15", "periodic_q15_f27", "walls_patches_q15_rk4",
                                  "walls_patches_q27_rk2", "periodic_q15_rk4", "periodic_q15_rk2iso",
                                  "walls_patches_q15_rk4iso"])
def test_adjoint_step_dot_product(case):
    """Per step: <lam, central difference of the step along d> (Richardson-
    extrapolated; measured 1e-12 .. 4e-9) equals <adjoint(lam), d> to 1e-8,
    h on D3Q15 / D3Q27 and
    the energy equation as the thermal LB on D3Q7 / 15 / 19 / 27 or RK2 / RK4
    (7-point or isotropic operators; the state then holds the T field)."""
    tag = case.split("_")[-1]
    thermal = {"f19": "D3Q19", "f15": "D3Q15", "f27": "D3Q27", "rk4": "RK4", "rk2": "RK2", "rk2iso": "RK2",
               "rk4iso": "RK4"}.get(tag, "D3Q7")
    q_phase = 27 if "_q27" in case else 15
    if case.startswith("walls_patches"):
        w = W.config5(n=16)
        w = w.replace(thermal=thermal, q_phase=q_phase)
    else:
        w = _periodic_case(q_phase, thermal)
    if tag.endswith("iso"):
        w = w.replace(params=W.Params(**dict(w.params.__dict__, rk_isotropic_fd=True)))
    d = gpu_domain(w)
    d.step(5)                                   # a state with flow and interface forces
    s = _state(d)
    rng = np.random.default_rng(11)
    lam = rng.standard_normal(s.size)
    dlt = rng.standard_normal(s.size) * (1e-2 * np.abs(s).max())
    def central(eps):
        out = []
        for sg in (1.0, -1.0):
            _set_state(d, s + sg * eps * dlt, w.q_phase, w.cells)
            d.step(1)
            out.append(_state(d))
        return lam @ ((out[0] - out[1]) / (2 * eps))

    # Richardson extrapolation of the central difference removes its
    # O(eps^2) truncation error (the step is nonlinear in the state)
    d1, d2 = central(2e-5), central(1e-5)
    lhs = (4.0 * d2 - d1) / 3.0
    _set_state(d, s, w.q_phase, w.cells)
    rhs = d.adjoint_step(lam) @ dlt
    print(case, lhs, rhs, abs(lhs - rhs) / abs(rhs), "plain central difference", abs(d2 - rhs) / abs(rhs))
    assert abs(lhs - rhs) <= 1e-8 * abs(rhs), (lhs, rhs)


def _oracle_J(w, steps):
    from harness import oracle_for
    o = oracle_for(w)
    o.step(steps)
    phi = o.macro()["phi"]
    z, y, x = np.meshgrid(np.arange(w.nz) + 0.5, np.arange(w.ny) + 0.5, np.arange(w.nx) + 0.5, indexing="ij")
    m = phi.sum()
    c = np.array([(phi * x).sum(), (phi * y).sum(), (phi * z).sum()]) / m
    return float(((c - np.array(w.target)) ** 2).sum())


@pytest.mark.parametrize("thermal", ["D3Q7", "D3Q19", "RK4", "RK2"])
def test_adjoint_gradient_matches_oracle_finite_differences(thermal):
    """16^3 adjoint workload (4 x 4 patches of 4 x 4 cells, walls), 40 steps,
    energy equation as the thermal LB on D3Q7 (the workload's) or D3Q19, or
    RK4 / RK2: GPU adjoint dJ/dI against central differences (h = 1e-4) of
    the FP64 oracle, every patch."""
    w = W.config5(n=16)
    if thermal != "D3Q7":
        w = w.replace(thermal=thermal)
    steps = 40
    d = gpu_domain(w)
    J, g = d.adjoint_run(steps, 10, w.target)
    assert abs(J - _oracle_J(w, steps)) <= 1e-11 * J
    h = 1e-4
    I0 = np.array(w.patches.intensity)
    fd = np.empty_like(I0)
    for k in range(len(I0)):
        Jp = _oracle_J(_with_intensity(w, I0 + h * np.eye(len(I0))[k]), steps)
        Jm = _oracle_J(_with_intensity(w, I0 - h * np.eye(len(I0))[k]), steps)
        fd[k] = (Jp - Jm) / (2 * h)
    err = np.abs(g - fd).max() / np.abs(fd).max()
    print("adjoint vs oracle FD", err, g[:4], fd[:4])
    assert err <= 1e-6


def test_adjoint_gradient_matches_complex_step_oracle():
    """16^3 adjoint workload, 200 steps with a checkpoint every 20: the GPU
    adjoint dJ/dI against the exact derivatives of the FP64 oracle
    (complex-step, one complex oracle run per patch;
    tests/golden/adjoint_cfg5_16cube_200steps.txt, written by
    tests/golden/make_adjoint_golden.py), to 1e-7 of max |dJ/dI|."""
    import os
    golden = np.loadtxt(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                     "adjoint_cfg5_16cube_200steps.txt"), comments="#")
    J_ref, g_ref = golden[0], golden[1:]
    w = W.config5(n=16)
    assert w.steps == 200
    d = gpu_domain(w)
    J, g = d.adjoint_run(200, 20, w.target)
    assert abs(J - J_ref) <= 1e-11 * J_ref
    err = np.abs(g - g_ref).max() / np.abs(g_ref).max()
    print("adjoint vs complex-step oracle", err)
    assert err <= 1e-7


@pytest.mark.parametrize("thermal", ["D3Q7", "RK4"])
def test_adjoint_checkpoint_spacing_is_exact(thermal):
    """Checkpoints every 1, 7 or 40 steps give the same J and gradient bit
    for bit (with RK the checkpoints carry the T field)."""
    w = W.config5(n=16).replace(thermal=thermal)
    res = []
    for K in (1, 7, 40):
        d = gpu_domain(w)
        res.append(d.adjoint_run(40, K, w.target))
        d.close()
    for J, g in res[1:]:
        assert J == res[0][0]
        assert np.array_equal(g, res[0][1])


def test_adjoint_gradient_full_size_vs_gpu_finite_differences():
    """64^3, 2000 steps, checkpoints every 100 (the adjoint workload): all 16
    components of dJ/dI against central differences (h = 1e-4) of the GPU
    FP64 forward.  With the normal cap 30 the error max |g - fd| / max |fd|
    is <= 1e-4.  The exact discrete adjoint (cap 0) is run too: over this
    horizon it grows far beyond the finite differences (its error is printed
    and must exceed 1, which is the measured divergence the cap removes)."""
    w = W.config5(n=64)
    h = 1e-4
    I0 = np.array(w.patches.intensity)

    def J_of(I):
        dd = gpu_domain(_with_intensity(w, I))
        dd.step(w.steps)
        m = dd.diagnostics()
        dd.close()
        c = np.array([m["mx"], m["my"], m["mz"]]) / m["mass"]
        return float(((c - np.array(w.target)) ** 2).sum())

    fd = np.empty_like(I0)
    for k in range(len(I0)):
        e = np.eye(len(I0))[k]
        fd[k] = (J_of(I0 + h * e) - J_of(I0 - h * e)) / (2 * h)
    d = gpu_domain(w)
    J, g = d.adjoint_run(w.steps, 100, w.target, normal_cap=30.0)
    d.close()
    assert abs(J - J_of(I0)) <= 1e-12 * J
    err = np.abs(g - fd).max() / np.abs(fd).max()
    print("capped adjoint (cap 30) vs GPU central differences, all 16:", f"{err:.3e}")
    assert err <= 1e-4
    d = gpu_domain(w)
    J0, g0 = d.adjoint_run(w.steps, 100, w.target, normal_cap=0.0)
    d.close()
    assert J0 == J
    err0 = np.abs(g0 - fd).max() / np.abs(fd).max()
    print("exact adjoint vs GPU central differences:", f"{err0:.3e}", "max |g|", f"{np.abs(g0).max():.3e}")
    assert not (err0 <= 1.0)      # diverged (or overflowed)


def test_capture_objective_autograd():
    import torch
    from paper_2401_03041_gb300 import lbm
    w = W.config5(n=16)

    def setup(I):
        return gpu_domain(_with_intensity(w, I))

    I = torch.tensor(w.patches.intensity, dtype=torch.float32, requires_grad=True)
    J = lbm.capture_objective(I, setup, 40, 10, w.target)
    J.backward()
    d = setup(w.patches.intensity)
    J_ref, g_ref = d.adjoint_run(40, 10, w.target)
    assert abs(J.item() - J_ref) <= 1e-6 * J_ref   # intensities round-tripped through float32
    assert np.allclose(I.grad.numpy(), g_ref, rtol=1e-5, atol=0)


@pytest.mark.parametrize("change", [{"alpha_H": 0.01}, {"rho_H": 3.0}])
def test_adjoint_rejects_conductivity_and_density_ratio(change):
    from paper_2401_03041_gb300 import lbm
    w = W.config5(n=16)
    w = w.replace(params=W.Params(**dict(w.params.__dict__, **change)))
    d = gpu_domain(w)
    with pytest.raises(lbm.LBMError) as e:
        d.adjoint_run(4, 2, w.target)
    assert e.value.status == -7
