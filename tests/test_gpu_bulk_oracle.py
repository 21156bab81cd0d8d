"""Multi-step oracle parity of the two tiled (tensor-TMA) step kernels, bulk
and skewed (the kernel the throughput benchmark times), in every storage
precision.

FP64: 200 steps on bulk-eligible lattices, every field and PDF set within
1e-11 relative of the FP64 oracle.

FP32 and FP16 storage (shifted PDFs, FP32 arithmetic): 200 steps of the
same kind of droplet workload on an 80-wide lattice (wide enough for the bulk
kernel in both), element by element against the FP64 oracle.  The errors are
printed (pytest -s) and bounded by the linear worst-case accumulation of the
storage rounding (tolerances derived in the comment above ``TOL``).
"""
import math

import numpy as np
import pytest

from harness import (gpu_domain, gpu_fields, gpu_state_in_oracle_order, oracle_for,
                     ragged_workload, relerr)

pytestmark = pytest.mark.gpu

STEPS = 200
TOL64 = 1e-11

# Bounds on the reduced-precision errors after STEPS steps.  phi and its
# mass follow from the storage rounding accumulated linearly (no damping
# assumed): phi = sum_i h_i with h stored as h_i - w_i/2, |h_i - w_i/2| <=
# w_i/2, so one step adds at most sum_i u_s w_i / 2 = u_s / 2 per cell (u_s
# the unit roundoff of the storage, 2^-24 FP32, 2^-11 FP16) plus a few 2^-24
# of FP32 arithmetic:
#   phi_abs  <= STEPS (u_s / 2 + 8 * 2^-24)    = 1.1e-4 (FP32), 5.0e-2 (FP16)
#   mass_rel <= STEPS (u_s / 2 + 8 * 2^-24) / mean(phi), mean(phi) ~ 0.1 here.
#   centroid <= L phi_abs / mean(phi) (L = 80, the box length)
#            = 0.09 lu (FP32); for FP16 this bound is vacuous (40 lu), and a
#              sanity bound of 0.5 lu is used instead.
# u, T and p* are small fields (|u| ~ 1e-3): the same absolute rounding is a
# larger relative error, so they get loose bounds and their measured values
# are printed.
TOL = {
    "fp32": {"phi_abs": 1.1e-4, "mass_rel": 1.1e-3, "u_l2_rel": 1e-2, "T_rel": 1e-2, "p_rel": 5e-2,
             "centroid": 0.09},
    "fp16": {"phi_abs": 5.0e-2, "mass_rel": 0.5, "u_l2_rel": 0.3, "T_rel": 0.3, "p_rel": 1.0,
             "centroid": 0.5},
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_03041_gb300 import build
    build.build()


_ORACLE = {}


def oracle_run(key, w):
    """The oracle's STEPS-step run of workload w (once per session)."""
    if key not in _ORACLE:
        o = oracle_for(w)
        o.step(STEPS)
        _ORACLE[key] = (o, o.macro(), o.diagnostics())
    return _ORACLE[key]


@pytest.mark.parametrize("kernel", ["bulk", "skew"])
@pytest.mark.parametrize("walls", [True, False])
def test_bulk_fp64_200_steps(walls, kernel):
    """40 x 24 x 16 (bulk-eligible in FP64: nx >= 36, ny >= 8), two moving
    droplets, heaters, gravity, unequal viscosities, walls or periodic z with
    a tilted gradient, D3Q7 thermal, 200 steps on the bulk kernel."""
    w = ragged_workload("D3Q7", 15, walls=walls, shape=(40, 24, 16))
    o, om_, _ = oracle_run(("fp64", walls), w)
    d = gpu_domain(w, kernel=kernel)
    d.step(STEPS)
    gf = gpu_fields(d)
    errs = {k: relerr(gf[k], om_[k]) for k in ("phi", "p", "T", "u")}
    st = gpu_state_in_oracle_order(d, w)
    ost = o.state()
    for k in st:
        errs["pdf_" + k] = relerr(st[k], ost[k])
    print(f"{kernel} fp64 200 steps walls={walls}", {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < TOL64, (k, v)


def reduced_precision_errors(d, om_, od):
    gf = gpu_fields(d)
    du = gf["u"] - om_["u"]
    gd = d.diagnostics()
    return {
        "phi_abs": float(np.abs(gf["phi"] - om_["phi"]).max()),
        "mass_rel": abs(gd["mass"] - od["mass"]) / abs(od["mass"]),
        "u_l2_rel": math.sqrt(float((du ** 2).sum()) / float((om_["u"] ** 2).sum())),
        "T_rel": relerr(gf["T"], om_["T"]),
        "p_rel": relerr(gf["p"], om_["p"]),
        "centroid": max(abs(a - b) for a, b in zip(gd["centroid"], od["centroid"])),
    }


@pytest.mark.parametrize("kernel", ["bulk", "skew"])
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_bulk_reduced_precision_200_steps_vs_oracle(precision, kernel):
    """80 x 24 x 16 walled droplet workload (bulk-eligible in FP32 and FP16
    storage), 200 steps of the bulk kernel against the FP64 oracle, element
    by element: phi L_inf, velocity L2, T and p* L_inf, phi mass, centroid."""
    w = ragged_workload("D3Q7", 15, walls=True, precision=precision, shape=(80, 24, 16))
    o, om_, od = oracle_run(("reduced", 80), w.replace(precision="fp64"))
    d = gpu_domain(w, kernel=kernel)
    d.step(STEPS)
    errs = reduced_precision_errors(d, om_, od)
    print(f"{kernel} {precision} 200 steps vs oracle", {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= TOL[precision][k], (precision, k, v, TOL[precision][k])
