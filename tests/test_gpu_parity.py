"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64: the GPU must match the oracle within 1e-11 relative (||.||_inf of the
difference over ||.||_inf of the oracle field, per field and per PDF set).
FP32 / FP16-storage: errors are measured and bounded loosely; the numbers are
printed (pytest -s) and recorded in the design notes.
"""
import math

import numpy as np
import pytest

import workloads as W
from harness import (bulk_fits, gpu_domain, gpu_fields, gpu_state_in_oracle_order,
                     load_state_into_gpu, oracle_for, ragged_workload, relerr, skew_fits)

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_03041_gb300 import build
    build.build()


def compare_all(d, o, w, tol, label=""):
    gf = gpu_fields(d)
    of = o.macro()
    errs = {k: relerr(gf[k], of[k]) for k in ("phi", "p", "T")}
    errs["u"] = relerr(gf["u"], of["u"])
    st = gpu_state_in_oracle_order(d, w)
    ost = o.state()
    for k in st:
        errs["pdf_" + k] = relerr(st[k], ost[k])
    print(label, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < tol, f"{label}: {k} relative error {v:.3e} >= {tol}"
    return errs


_CFG1 = {}


def config1_oracle():
    """The oracle's 200-step config-1 run (computed once per session)."""
    if not _CFG1:
        w = W.config1()
        o = oracle_for(w)
        o.step(w.steps)
        _CFG1["o"] = o
    return _CFG1["o"]


def test_config1_fp64_200_steps():
    """32^3 periodic droplet, D3Q15 phase field, D3Q7 thermal, 200 steps."""
    w = W.config1()
    d = gpu_domain(w)
    d.step(w.steps)
    compare_all(d, config1_oracle(), w, TOL64, "config1 fp64 200 steps")


def _kernels(precision, q_phase, thermal):
    ks = ["generic"]
    if bulk_fits(precision, q_phase, thermal):
        ks.append("bulk")
    if skew_fits(precision, q_phase, thermal):
        ks.append("skew")
    return ks


@pytest.mark.parametrize("thermal", ["D3Q7", "D3Q15", "D3Q19", "D3Q27", "RK2", "RK4"])
@pytest.mark.parametrize("q_phase", [15, 27])
def test_ragged_walls_fp64(thermal, q_phase):
    """40 x 20 x 13 (ragged against both kernels' tiles), walls, heaters, two
    moving droplets, every energy solver and both phase-field stencils, on
    the generic kernel and on the bulk (tensor-TMA) one."""
    w = ragged_workload(thermal, q_phase, walls=True)
    o = oracle_for(w)
    o.step(12)
    for kern in _kernels("fp64", q_phase, thermal):
        d = gpu_domain(w, kernel=kern)
        d.step(12)
        compare_all(d, o, w, TOL64, f"ragged walls {thermal} q{q_phase} {kern}")


@pytest.mark.parametrize("thermal,q_phase", [("D3Q7", 15), ("D3Q15", 15), ("D3Q19", 15), ("RK2", 15), ("RK4", 15),
                                             ("D3Q27", 15), ("D3Q7", 27), ("D3Q27", 27)])
def test_ragged_periodic_fp64(thermal, q_phase):
    """Periodic in x, y and z: every ghost side the tiled kernels read, for
    each stencil of h, g and f (the ghost fill refreshes only those)."""
    w = ragged_workload(thermal, q_phase, walls=False)
    o = oracle_for(w)
    o.step(12)
    for kern in _kernels("fp64", q_phase, thermal):
        d = gpu_domain(w, kernel=kern)
        d.step(12)
        compare_all(d, o, w, TOL64, f"ragged periodic {thermal} q{q_phase} {kern}")


@pytest.mark.parametrize("kernel", ["bulk", "skew"])
@pytest.mark.parametrize("thermal", ["D3Q7", "D3Q15", "RK4"])
@pytest.mark.parametrize("walls", [True, False])
def test_bulk_multi_tile_chunked_fp64(walls, thermal, kernel, monkeypatch):
    """72 x 24 x 20: several tiles in x (ragged) and y, the z range split
    into chunks of 6 planes (pipeline prologue at every chunk start, a last
    chunk of 2 planes); D3Q15 thermal runs the one-stage g ring."""
    if kernel == "skew" and not skew_fits("fp64", 15, thermal):
        pytest.skip("layout does not fit")
    monkeypatch.setenv("LBM_ZCHUNK", "6")
    w = ragged_workload(thermal, 15, walls=walls, shape=(72, 24, 20))
    o = oracle_for(w)
    o.step(10)
    d = gpu_domain(w, kernel=kernel)
    assert d.kernel_info()["grid"][2] == 4
    d.step(10)
    compare_all(d, o, w, TOL64, f"{kernel} chunked walls={walls} {thermal}")


@pytest.mark.parametrize("kernel", ["bulk", "skew"])
@pytest.mark.parametrize("nx,ny", [(74, 16), (75, 16), (75, 18)])
def test_bulk_ghost_fill_paths_fp64(nx, ny, kernel):
    """Periodic in x and y with nx a multiple of the 16-byte vector width but
    not of two vectors (74) or not of one (75): the two slower ghost-fill
    paths; with ny a multiple of the tile rows or not (18, a last tile row
    half outside the lattice); against the oracle."""
    w = ragged_workload("D3Q7", 15, walls=False, shape=(nx, ny, 8))
    o = oracle_for(w)
    o.step(8)
    d = gpu_domain(w, kernel=kernel)
    d.step(8)
    compare_all(d, o, w, TOL64, f"{kernel} ghost paths nx={nx} ny={ny}")


@pytest.mark.parametrize("kernel", ["bulk", "skew"])
@pytest.mark.parametrize("precision,nx,ny", [("fp32", 76, 16), ("fp32", 78, 16), ("fp32", 78, 18),
                                             ("fp16", 88, 16), ("fp16", 84, 16), ("fp16", 84, 18)])
def test_bulk_ghost_fill_paths_reduced_precision(precision, nx, ny, kernel):
    """The same ghost-fill paths in FP32 / FP16 storage: the tiled kernels
    equal the generic one to the storage rounding after 12 periodic steps."""
    w = ragged_workload("D3Q7", 15, walls=False, precision=precision, shape=(nx, ny, 8))
    a = gpu_domain(w, kernel="generic")
    b = gpu_domain(w, kernel=kernel)
    a.step(12)
    b.step(12)
    fa, fb = gpu_fields(a), gpu_fields(b)
    tol = 1e-5 if precision == "fp32" else 1e-2
    for k in ("phi", "u", "p", "T"):
        e = relerr(fb[k], fa[k])
        assert e < tol, (precision, nx, k, e)


@pytest.mark.parametrize("thermal,q_phase", [("D3Q19", 15), ("D3Q27", 15), ("D3Q7", 27)])
def test_tiled_equals_generic_periodic_fp32(thermal, q_phase):
    """Periodic FP32 lattices with the larger stencils: the library's tiled
    kernel (skewed, or bulk where the skewed layout does not fit) equals the
    generic one to the storage rounding after 20 steps, so every ghost side it
    reads is refreshed."""
    w = ragged_workload(thermal, q_phase, walls=False, precision="fp32", shape=(80, 24, 12))
    a = gpu_domain(w, kernel="generic")
    b = gpu_domain(w)
    assert b.kernel_info()["kernel"] in ("bulk", "skew"), b.kernel_info()
    a.step(20)
    b.step(20)
    fa, fb = gpu_fields(a), gpu_fields(b)
    for k in ("phi", "u", "p", "T"):
        e = relerr(fb[k], fa[k])
        print(thermal, q_phase, b.kernel_info()["kernel"], k, f"{e:.2e}")
        assert e < 1e-5, (k, e)


@pytest.mark.parametrize("kernel", ["bulk", "skew"])
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("thermal", ["D3Q7", "D3Q15", "RK2"])
def test_bulk_equals_generic_reduced_precision(precision, thermal, kernel):
    """The kernels compute the same arithmetic: in FP32 / FP16 storage they
    agree to the storage rounding after 20 steps."""
    if kernel == "skew" and not skew_fits(precision, 15, thermal):
        pytest.skip("layout does not fit")
    w = ragged_workload(thermal, 15, walls=True, precision=precision, shape=(80, 24, 12))
    a = gpu_domain(w, kernel="generic")
    b = gpu_domain(w, kernel=kernel)
    a.step(20)
    b.step(20)
    fa, fb = gpu_fields(a), gpu_fields(b)
    tol = 1e-5 if precision == "fp32" else 1e-2
    for k in ("phi", "u", "p", "T"):
        e = relerr(fb[k], fa[k])
        print(precision, thermal, k, f"{e:.2e}")
        assert e < tol, (k, e)


@pytest.mark.parametrize("thermal", ["D3Q19", "RK2"])
def test_perturbed_state_one_step_fp64(thermal):
    """Arbitrary non-equilibrium PDFs (equilibrium + seeded noise in every
    direction) exercise every term of the collisions in one step."""
    w = ragged_workload(thermal, 27, walls=True)
    o = oracle_for(w)
    o.step(3)
    st = o.state()
    rng = np.random.Generator(np.random.PCG64(77))
    for k in st:
        st[k] = st[k] + rng.standard_normal(st[k].shape) * 1e-4
    o.h, o.g = st["h"], st["g"]
    if "f" in st:
        o.f = st["f"]
    else:
        o.T = st["T"]
    d = gpu_domain(w)
    load_state_into_gpu(d, w, st)
    compare_all(d, o, w, 1e-14 * 1e3, "perturbed, before step")
    d.step(1)
    o.step(1)
    compare_all(d, o, w, TOL64, f"perturbed one step {thermal}")


def test_rk_isotropic_operator_and_patches_fp64():
    w = ragged_workload("RK4", 15, walls=True)
    w = w.replace(params=W.Params(**{**w.params.__dict__, "rk_isotropic_fd": True}),
                  patches=W.HeaterPatches(z=0, sx=10, sy=5, x0=[0, 10, 20, 30], y0=[0, 5, 10, 15],
                                          intensity=[0.1, 0.2, 0.05, 0.3]))
    d = gpu_domain(w)
    o = oracle_for(w)
    d.step(8)
    o.step(8)
    compare_all(d, o, w, TOL64, "rk4 iso + patches")


def _ratio_workload(thermal, walls=True, iso=False):
    w = ragged_workload(thermal, 15, walls=walls)
    kw = dict(w.params.__dict__, alpha_L=0.1, alpha_H=0.02, rk_isotropic_fd=iso)
    return w.replace(params=W.Params(**kw))


@pytest.mark.parametrize("thermal,walls,iso", [("D3Q7", True, False), ("D3Q19", True, False),
                                               ("D3Q15", False, False), ("RK2", True, False),
                                               ("RK4", True, False), ("RK4", False, True)])
def test_conductivity_ratio_fp64(thermal, walls, iso):
    """alpha_H = alpha_L / 5 (Sec. 2.3, kappa linear in phi): per-cell LB rate
    and background source, or the RK grad alpha term in stage 1 (step kernel)
    and stages 2..4 (stage kernel, phi of the step); with a tilted background
    gradient, walls or periodic z, generic and bulk kernels."""
    w = _ratio_workload(thermal, walls, iso)
    o = oracle_for(w)
    o.step(12)
    for kern in _kernels("fp64", 15, thermal):
        d = gpu_domain(w, kernel=kern)
        d.step(12)
        compare_all(d, o, w, TOL64, f"conductivity ratio {thermal} walls={walls} iso={iso} {kern}")


@pytest.mark.parametrize("thermal,walls,iso,case",
                         [("D3Q7", True, False, "cp"), ("D3Q19", False, False, "cp"),
                          ("D3Q27", True, False, "cp_rho"), ("RK4", True, False, "cp"),
                          ("RK2", False, True, "cp_rho"), ("D3Q15", True, False, "uniform"),
                          ("RK4", False, False, "uniform")])
def test_heat_capacity_ratio_fp64(thermal, walls, iso, case):
    """Heat capacity rho c_p of Eq. temperature with c_p linear in phi
    (Sec. 2.3): c_p,H / c_p,L = 3 with a conductivity ratio 1/5 ("cp"), also
    with rho_H / rho_L = 4 entering rho c_p ("cp_rho"), or a uniform
    rho c_p = 3 that only rescales the diffusivity ("uniform"): per-cell LB
    rate with the background and grad(rho c_p) sources, or the RK right-hand
    side divided by rho c_p; generic and tiled kernels match the oracle
    within 1e-11 after 12 steps."""
    w = ragged_workload(thermal, 15, walls=walls)
    kw = dict(w.params.__dict__, rk_isotropic_fd=iso)
    if case == "uniform":
        kw.update(cp_L=3.0, cp_H=3.0, alpha_L=0.15, alpha_H=0.15)
    else:
        kw.update(cp_L=1.0, cp_H=3.0, alpha_L=0.1, alpha_H=0.02)
        if case == "cp_rho":
            kw.update(rho_L=1.0, rho_H=4.0)
    w = w.replace(params=W.Params(**kw))
    o = oracle_for(w)
    o.step(12)
    for kern in _kernels("fp64", 15, thermal):
        d = gpu_domain(w, kernel=kern)
        d.step(12)
        compare_all(d, o, w, TOL64, f"heat capacity {case} {thermal} walls={walls} iso={iso} {kern}")


@pytest.mark.parametrize("thermal,ratio", [("D3Q7", False), ("D3Q19", True), ("RK4", True), ("RK2", False)])
def test_modulated_bottom_wall_fp64(thermal, ratio):
    """Bottom wall at T_bottom + 0.3 cos(2 pi 2 (x + 1/2) / nx) (the heated
    channel's wall): anti-bounce-back, the Dirichlet ghosts of the stencils
    and the initial conduction profile all take the column's wall value."""
    w = _ratio_workload(thermal) if ratio else ragged_workload(thermal, 15, walls=True)
    w = w.replace(params=W.Params(**dict(w.params.__dict__, T_bottom_amp=0.3, T_bottom_waves=2)))
    o = oracle_for(w)
    o.step(10)
    for kern in _kernels("fp64", 15, thermal):
        d = gpu_domain(w, kernel=kern)
        d.step(10)
        compare_all(d, o, w, TOL64, f"modulated wall {thermal} ratio={ratio} {kern}")


def _density_workload(thermal, walls=True, q_phase=15, ratio=10.0, shape=(40, 20, 13), alpha_ratio=False):
    w = ragged_workload(thermal, q_phase, walls=walls, shape=shape)
    kw = dict(w.params.__dict__, rho_L=1.0, rho_H=ratio)
    if alpha_ratio:
        kw.update(alpha_L=0.1, alpha_H=0.02)
    return w.replace(params=W.Params(**kw))


@pytest.mark.parametrize("thermal,walls,q_phase,alpha_ratio",
                         [("D3Q7", True, 15, False), ("D3Q19", False, 15, False), ("RK4", True, 27, False),
                          ("D3Q15", True, 15, True), ("RK2", False, 15, True), ("D3Q27", True, 27, False)])
def test_density_ratio_fp64(thermal, walls, q_phase, alpha_ratio):
    """rho_H / rho_L = 10 (Sec. 2.2 pressure and viscous correction forces,
    strain from the non-equilibrium moments of g), unequal viscosities,
    gravity, moving droplets, with and without a conductivity ratio, walls
    or periodic z, both phase-field stencils: generic and bulk kernels match
    the oracle within 1e-11 after 12 steps."""
    w = _density_workload(thermal, walls, q_phase, alpha_ratio=alpha_ratio)
    o = oracle_for(w)
    o.step(12)
    for kern in _kernels("fp64", q_phase, thermal):
        d = gpu_domain(w, kernel=kern)
        d.step(12)
        compare_all(d, o, w, TOL64, f"density ratio {thermal} walls={walls} q{q_phase} {kern}")


@pytest.mark.parametrize("walls", [True, False])
def test_density_ratio_bulk_fp64_60_steps(walls):
    """The bulk kernel's density-ratio path (second exchange between its two
    roles) over 60 steps on a 72-wide lattice."""
    w = _density_workload("D3Q7", walls, shape=(72, 24, 20))
    o = oracle_for(w)
    o.step(60)
    d = gpu_domain(w, kernel="bulk")
    d.step(60)
    compare_all(d, o, w, TOL64, f"density ratio bulk 60 steps walls={walls}")


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-4), ("fp16", 5e-2)])
def test_density_ratio_reduced_precision(precision, tol):
    """FP32 / FP16-storage density-ratio runs (bulk kernel) stay within the
    reduced-precision error of the FP64 run after 40 steps."""
    w = _density_workload("D3Q7", True, shape=(88, 24, 12))
    ref = gpu_domain(w)
    ref.step(40)
    d = gpu_domain(w, precision=precision, kernel="bulk")
    d.step(40)
    a, b = gpu_fields(d), gpu_fields(ref)
    for k in ("phi", "T"):
        assert relerr(a[k], b[k]) < tol, (precision, k, relerr(a[k], b[k]))


def _wall_workload(thermal, q_phase=15, moving=True, wetting=True, alpha_ratio=False, shape=(40, 20, 13)):
    w = ragged_workload(thermal, q_phase, walls=True, shape=shape)
    kw = dict(w.params.__dict__)
    if moving:
        kw.update(wall_u_top=(0.02, -0.01), wall_u_bottom=(-0.005, 0.01))
    if wetting:
        kw.update(theta_bottom=60.0, theta_top=130.0)
    if alpha_ratio:
        kw.update(alpha_L=0.1, alpha_H=0.02)
    return w.replace(params=W.Params(**kw))


@pytest.mark.parametrize("thermal,q_phase,moving,wetting,alpha_ratio",
                         [("D3Q7", 15, True, True, False), ("D3Q19", 27, True, False, False),
                          ("RK4", 15, False, True, True), ("D3Q15", 15, True, True, True),
                          ("RK2", 27, True, True, False), ("D3Q27", 15, True, True, False)])
def test_moving_walls_and_wetting_fp64(thermal, q_phase, moving, wetting, alpha_ratio):
    """Sheared channel walls (tangential velocities on both walls) and
    contact angles 60 / 130 degrees, with moving droplets near the walls,
    every energy solver, both phase-field stencils: all kernels match the
    oracle within 1e-11 after 12 steps."""
    w = _wall_workload(thermal, q_phase, moving, wetting, alpha_ratio)
    o = oracle_for(w)
    o.step(12)
    for kern in _kernels("fp64", q_phase, thermal):
        d = gpu_domain(w, kernel=kern)
        d.step(12)
        compare_all(d, o, w, TOL64, f"walls {thermal} q{q_phase} moving={moving} wetting={wetting} {kern}")


@pytest.mark.parametrize("kernel", ["bulk", "skew"])
def test_moving_walls_and_wetting_tiled_fp64_60_steps(kernel):
    """The tiled kernels' wall rules over 60 steps on a 72-wide lattice."""
    w = _wall_workload("D3Q7", shape=(72, 24, 20))
    o = oracle_for(w)
    o.step(60)
    d = gpu_domain(w, kernel=kernel)
    d.step(60)
    compare_all(d, o, w, TOL64, f"walls 60 steps {kernel}")


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-4), ("fp16", 5e-2)])
def test_conductivity_ratio_reduced_precision(precision, tol):
    """FP32 / FP16-storage runs of the ratio workload (D3Q7 and RK4) stay
    within the reduced-precision error of the FP64 GPU run after 40 steps."""
    for thermal in ("D3Q7", "RK4"):
        w = _ratio_workload(thermal)
        ref = gpu_domain(w)
        ref.step(40)
        d = gpu_domain(w, precision=precision)
        d.step(40)
        a, b = gpu_fields(d), gpu_fields(ref)
        for k in ("phi", "T"):
            assert relerr(a[k], b[k]) < tol, (precision, thermal, k, relerr(a[k], b[k]))


def _field_tensor(q, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(q).ravel(), dtype=dtype, device="cuda")


@pytest.mark.parametrize("thermal,fdtype", [("D3Q7", "f64"), ("D3Q19", "f32"), ("RK4", "f32"),
                                            ("RK2", "f64")])
def test_heater_field_fp64(thermal, fdtype):
    """lbm_set_heater_field: a seeded per-cell heat field (Gaussian spots plus
    noise) on top of the Gaussian sources, FP64 state, FP64 or FP32 field (the
    oracle gets the FP32-rounded values), generic and bulk kernels."""
    import torch
    w = ragged_workload(thermal, 15, walls=True)
    q = W.heater_field(3, (w.nz, w.ny, w.nx))
    if fdtype == "f32":
        q = q.astype(np.float32).astype(np.float64)
    o = oracle_for(w)
    o.add_heat_field(q)
    o.step(12)
    qt = _field_tensor(q, torch.float64 if fdtype == "f64" else torch.float32)
    for kern in _kernels("fp64", 15, thermal):
        d = gpu_domain(w, kernel=kern)
        d.set_heater_field(qt)
        d.step(12)
        compare_all(d, o, w, TOL64, f"heater field {thermal} {fdtype} {kern}")


def test_heater_field_equals_patches_and_rejects_bad_pointers():
    """A field holding the heater patches' values gives bit for bit the run
    with the patches; removing the field restores the plain run; host,
    misaligned pointers and unknown dtypes are rejected."""
    import ctypes

    import torch
    from paper_2401_03041_gb300 import lbm
    w = ragged_workload("D3Q7", 15, walls=True, precision="fp32", shape=(80, 24, 12))
    pw = w.replace(patches=W.HeaterPatches(z=2, sx=9, sy=5, x0=[3, 40], y0=[2, 12],
                                           intensity=[0.03, 0.07]))
    box = np.zeros((w.nz, w.ny, w.nx))
    for k in range(2):
        box[2, pw.patches.y0[k]:pw.patches.y0[k] + 5, pw.patches.x0[k]:pw.patches.x0[k] + 9] = \
            pw.patches.intensity[k]
    a = gpu_domain(pw)
    a.step(9)
    b = gpu_domain(w)
    b.set_heater_field(_field_tensor(box, torch.float64))
    b.step(9)
    fa, fb = gpu_fields(a), gpu_fields(b)
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    c = gpu_domain(w)
    c.set_heater_field(_field_tensor(box, torch.float32))
    c.set_heater_field(None)
    c.step(9)
    e = gpu_domain(w)
    e.step(9)
    fc, fe = gpu_fields(c), gpu_fields(e)
    assert not np.array_equal(fa["T"], fe["T"])
    for k in fc:
        assert np.array_equal(fc[k], fe[k]), k
    L = lbm.lib()
    host = np.zeros(w.cells)
    assert L.lbm_set_heater_field(e._h, ctypes.c_void_p(host.ctypes.data), 0) == -1
    dev = _field_tensor(box, torch.float64)
    assert L.lbm_set_heater_field(e._h, ctypes.c_void_p(dev.data_ptr() + 4), 0) == -1
    assert L.lbm_set_heater_field(e._h, ctypes.c_void_p(dev.data_ptr()), 2) == -1
    assert L.lbm_set_heater_field(e._h, ctypes.c_void_p(dev.data_ptr()), 0) == 0


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 1, 2), (33, 9, 1), (5, 17, 3)])
def test_tiny_and_degenerate_lattices_fp64(shape):
    nx, ny, nz = shape
    p = W.Params(grad_T=(1e-3, 0, 0), grad_T_origin=(nx / 2, ny / 2, nz / 2))
    w = W.Workload("tiny", nx, ny, nz, 5, p, [W.Droplet(nx / 2, ny / 2, nz / 2, 1.5, 1e-3, 0, 0)],
                   q_phase=15, thermal="D3Q7", precision="fp64")
    d = gpu_domain(w)
    o = oracle_for(w)
    d.step(5)
    o.step(5)
    compare_all(d, o, w, TOL64, f"tiny {shape}")


def test_no_droplets_and_walls_nz2_fp64():
    p = W.Params(walls_z=True, T_bottom=-1.0, T_top=1.0)
    w = W.Workload("empty", 8, 8, 2, 5, p, [], q_phase=15, thermal="D3Q15", precision="fp64")
    d = gpu_domain(w)
    o = oracle_for(w)
    d.step(7)
    o.step(7)
    compare_all(d, o, w, TOL64, "no droplets nz=2")


def test_diagnostics_fp64():
    w = ragged_workload("D3Q7", 15, walls=True)
    d = gpu_domain(w)
    o = oracle_for(w)
    d.step(4)
    o.step(4)
    gd = d.diagnostics()
    od = o.diagnostics()
    for k in ("mass", "heat", "kinetic", "mx", "my", "mz"):
        assert abs(gd[k] - od[k]) <= 1e-11 * max(abs(od[k]), 1e-30), (k, gd[k], od[k])
    assert gd["level"] == 4
    # fused into the step: the level the step consumed
    sd = d.step_diagnostics(1)
    assert sd["level"] == 4 and abs(sd["mass"] - gd["mass"]) <= 1e-13 * abs(gd["mass"])
    assert d.level() == 5


def test_mass_conserved_fp64_long():
    w = ragged_workload("D3Q7", 15, walls=True)
    d = gpu_domain(w)
    m0 = d.diagnostics()["mass"]
    d.step(500)
    m1 = d.diagnostics()["mass"]
    assert abs(m1 - m0) / m0 < 1e-12


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-4), ("fp16", 5e-2)])
def test_config1_reduced_precision_error(precision, tol):
    """FP32 / FP16-storage against the FP64 oracle on config 1 (200 steps):
    phi L_inf, velocity L2 (relative), phi mass and centroid."""
    w = W.config1()
    d = gpu_domain(w, precision)
    d.step(w.steps)
    o = config1_oracle()
    gf = gpu_fields(d)
    of = o.macro()
    phi_inf = relerr(gf["phi"], of["phi"])
    du = gf["u"] - of["u"]
    u_l2 = math.sqrt((du ** 2).sum() / (of["u"] ** 2).sum())
    gd, od = d.diagnostics(), o.diagnostics()
    mass = abs(gd["mass"] - od["mass"]) / od["mass"]
    cen = max(abs(a - b) for a, b in zip(gd["centroid"], od["centroid"]))
    print(f"{precision}: phi_inf={phi_inf:.3e} u_L2={u_l2:.3e} mass={mass:.3e} centroid={cen:.3e}")
    assert phi_inf < tol
    assert mass < tol
    assert cen < 1e-2


def test_full_size_sampled_fp32():
    """512^3 periodic, 64 droplets (the throughput workload), FP32, in the
    launch configuration the benchmark times: after one step, a 20^3 sample
    cut across a droplet interface matches an oracle run on the surrounding
    28^3 box (periodic wrap garbage stays > 2 cells from the sample)."""
    import torch
    w = W.config4("D3Q7", "fp32")
    d = gpu_domain(w, kernel="skew")
    m0 = d.diagnostics()["mass"]
    d.step(1)
    gf = d.fields(dtype="f32")
    # a droplet whose sample box does not cross the periodic boundary (the
    # background temperature term G.(x - x0) uses unwrapped coordinates)
    def centre(dr):
        return [int(round(dr.cx + dr.R)), int(round(dr.cy)), int(round(dr.cz))]
    drop = next(dr for dr in w.droplets
                if all(14 <= v <= n - 15 for v, n in zip(centre(dr), (w.nx, w.ny, w.nz))))
    c = centre(drop)
    lo = [v - 14 for v in c]
    idx = [np.arange(l, l + 28) % n for l, n in zip(lo, (w.nx, w.ny, w.nz))]
    from oracle import model as om
    o = om.build(w, origin=tuple(lo), shape=(28, 28, 28))
    o.step(1)
    of = o.macro()
    inner = (slice(4, 24),) * 3
    for name in ("phi", "p", "T", "u"):
        g = gf[name].detach().cpu().numpy()
        if name == "u":
            sub = g[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
            ref = of["u"][(slice(None),) + inner]
            got = sub[(slice(None),) + inner]
        else:
            sub = g[idx[2]][:, idx[1]][:, :, idx[0]]
            ref = of[name][inner]
            got = sub[inner]
        e = relerr(got, ref)
        print("512^3 sample", name, f"{e:.2e}")
        assert e < (1e-4 if name != "T" else 1e-2)
    m1 = d.diagnostics()["mass"]
    assert abs(m1 - m0) / m0 < 1e-6
    del d
    torch.cuda.empty_cache()
