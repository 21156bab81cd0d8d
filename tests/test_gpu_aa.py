"""The in-place (AA-pattern) PDF layout: one PDF set per field, updated in
place by alternating a gather-from-neighbours step and a local step, with a
(phi, T) field of each level for the finite differences.

Two implementations: the generic tiles ('aa', every model extension) and the
skewed kernel's tensor-TMA tiles ('aa_tiled', every extension but the
density ratio, with the periodic ghosts refreshed before and folded back
after each step from an even level).

FP64: equal to the generic two-grid kernel to rounding (fields and the
populations p_i(x) returned by lbm_get_pdfs, after an odd and an even number
of steps, within 1e-12 of each field's magnitude: the kernels are compiled
separately and contract their products into FMAs differently) on workloads
that exercise every wall rule and extension, and within 1e-11 of the oracle
after 200 steps.  FP32 / FP16 storage: within the reduced-precision bounds of
the tiled kernels against the FP64 oracle.  Checkpoints resume bit for bit,
the layout is recorded in the state, and the workspace is about half.
"""
import numpy as np
import pytest

import workloads as W
from harness import gpu_domain, gpu_fields, gpu_state_in_oracle_order, oracle_for, ragged_workload, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_03041_gb300 import build
    build.build()


def _variant(name):
    if name == "walls_moving_wetting":
        w = ragged_workload("D3Q7", 15, walls=True)
        return w.replace(params=W.Params(**dict(w.params.__dict__, wall_u_top=(0.02, -0.01),
                                                wall_u_bottom=(-0.005, 0.01), theta_bottom=60.0,
                                                theta_top=130.0)))
    if name == "periodic_d3q19_q27":
        return ragged_workload("D3Q19", 27, walls=False)
    if name == "rk4_conductivity_ratio":
        w = ragged_workload("RK4", 15, walls=True)
        return w.replace(params=W.Params(**dict(w.params.__dict__, alpha_L=0.1, alpha_H=0.02)))
    if name == "density_ratio_d3q15":
        w = ragged_workload("D3Q15", 15, walls=True)
        return w.replace(params=W.Params(**dict(w.params.__dict__, rho_L=1.0, rho_H=10.0)))
    if name == "d3q7_heat_capacity_ratio":
        w = ragged_workload("D3Q7", 15, walls=True)
        return w.replace(params=W.Params(**dict(w.params.__dict__, alpha_L=0.1, alpha_H=0.02, cp_L=1.0,
                                                cp_H=3.0)))
    if name == "rk2_periodic_heaters":
        return ragged_workload("RK2", 15, walls=False)
    raise KeyError(name)


def _uniform_variant(name):
    if name == "modulated_wall_d3q19":
        w = ragged_workload("D3Q19", 15, walls=True)
        return w.replace(params=W.Params(**dict(w.params.__dict__, T_bottom_amp=0.3, T_bottom_waves=2,
                                                wall_u_bottom=(0.01, 0.005))))
    if name == "walls_d3q7":
        return ragged_workload("D3Q7", 15, walls=True)
    if name == "periodic_d3q15_q27":
        return ragged_workload("D3Q15", 27, walls=False)
    if name == "walls_rk4":
        return ragged_workload("RK4", 15, walls=True)
    if name == "periodic_d3q27":
        return ragged_workload("D3Q27", 15, walls=False)
    return _variant(name)


@pytest.mark.parametrize("kernel,name", [("aa", n) for n in ("walls_moving_wetting", "periodic_d3q19_q27",
                                                             "rk4_conductivity_ratio", "d3q7_heat_capacity_ratio",
                                                             "density_ratio_d3q15", "rk2_periodic_heaters")]
                         + [("aa_tiled", n) for n in ("walls_d3q7", "periodic_d3q19_q27", "periodic_d3q15_q27",
                                                      "walls_rk4", "rk2_periodic_heaters", "periodic_d3q27",
                                                      "walls_moving_wetting", "rk4_conductivity_ratio",
                                                      "d3q7_heat_capacity_ratio", "modulated_wall_d3q19")])
def test_aa_equals_two_grid_fp64(kernel, name):
    """40 x 20 x 13 (ragged against the tiles in x and y): both in-place
    implementations against the generic two-grid kernel after an odd (7) and
    an even (13) number of steps."""
    w = _uniform_variant(name)
    a = gpu_domain(w, kernel=kernel)
    b = gpu_domain(w, kernel="generic")
    for steps in (7, 6):          # odd level 7, then even level 13
        a.step(steps)
        b.step(steps)
        fa, fb = gpu_fields(a), gpu_fields(b)
        for k in fa:
            e = relerr(fa[k], fb[k])
            assert e <= 1e-12, (name, k, a.level(), e)
        sa, sb = gpu_state_in_oracle_order(a, w), gpu_state_in_oracle_order(b, w)
        for k in sa:
            e = relerr(sa[k], sb[k])
            assert e <= 1e-12, (name, k, a.level(), e)
    da, db = a.diagnostics(), b.diagnostics()
    assert abs(da["mass"] - db["mass"]) <= 1e-12 * abs(db["mass"])
    assert abs(da["kinetic"] - db["kinetic"]) <= 1e-10 * abs(db["kinetic"])


@pytest.mark.parametrize("kernel", ["aa", "aa_tiled"])
def test_aa_fp64_200_steps_vs_oracle(kernel):
    w = ragged_workload("D3Q7", 15, walls=True, shape=(40, 24, 16))
    o = oracle_for(w)
    o.step(200)
    d = gpu_domain(w, kernel=kernel)
    d.step(200)
    gf, om_ = gpu_fields(d), o.macro()
    errs = {k: relerr(gf[k], om_[k]) for k in ("phi", "p", "T", "u")}
    st, ost = gpu_state_in_oracle_order(d, w), o.state()
    for k in st:
        errs["pdf_" + k] = relerr(st[k], ost[k])
    print(kernel, "fp64 200 steps", {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < 1e-11, (k, v)


@pytest.mark.parametrize("kernel,precision,tol_phi", [("aa", "fp32", 1.1e-4), ("aa", "fp16", 5e-2),
                                                     ("aa_tiled", "fp32", 1.1e-4), ("aa_tiled", "fp16", 5e-2)])
def test_aa_reduced_precision_matches_two_grid(kernel, precision, tol_phi):
    """Reduced-precision storage in the in-place layout: after 60 steps both
    the in-place and the generic two-grid kernel stay within the FP64
    oracle's phi bound for that storage (the two round differently where the
    compiler contracts differently, so they are not compared bit for bit).
    88 x 20 x 13: wide enough for the tiles in FP16 (rows of 80 or more)."""
    w = ragged_workload("D3Q7", 15, walls=True, precision=precision, shape=(88, 20, 13))
    a = gpu_domain(w, kernel=kernel)
    b = gpu_domain(w, kernel="generic")
    a.step(60)
    b.step(60)
    fa, fb = gpu_fields(a), gpu_fields(b)
    o = oracle_for(w.replace(precision="fp64"))
    o.step(60)
    ea = np.abs(fa["phi"] - o.macro()["phi"]).max()
    eb = np.abs(fb["phi"] - o.macro()["phi"]).max()
    print(precision, "phi error in place", ea, "two-grid", eb)
    assert ea < tol_phi and eb < tol_phi


def test_aa_tiled_falls_back_for_density_ratio():
    """The tiled in-place kernels cover every model extension but the density
    ratio (its forces need the moments and the stencils of one plane
    together), which runs the in-place step on the generic tiles."""
    w = ragged_workload("D3Q7", 15, walls=True)
    d = gpu_domain(w, kernel="aa_tiled")
    d.set_params(W.Params(**dict(w.params.__dict__, wall_u_top=(0.01, 0.0), theta_top=60.0, alpha_H=0.02)))
    assert d.kernel_info()["kernel"] == "aa_tiled"
    d.set_params(W.Params(**dict(w.params.__dict__, rho_H=4.0)))
    assert d.kernel_info()["kernel"] == "aa"
    d.set_params(w.params)
    assert d.kernel_info()["kernel"] == "aa_tiled"


@pytest.mark.parametrize("kernel", ["aa", "aa_tiled"])
def test_aa_checkpoint_resume_and_layout_check(kernel):
    from paper_2401_03041_gb300 import lbm
    w = ragged_workload("D3Q15", 15, walls=True)
    a = gpu_domain(w, kernel=kernel)
    a.step(5)                          # odd level
    blob = a.save_state()
    a.step(4)
    ref = gpu_fields(a)
    b = gpu_domain(w, kernel=kernel)
    b.load_state(blob)
    assert b.level() == 5
    b.step(4)
    got = gpu_fields(b)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k
    c = gpu_domain(w, kernel="generic")
    with pytest.raises(lbm.LBMError):
        c.load_state(blob)            # a state of the in-place layout
    with pytest.raises(lbm.LBMError):
        a.adjoint_run(2, 1, (0.0, 0.0, 0.0))
