"""Physics pins of the FP64 oracle: what the paper's model must reproduce
whatever the implementation (closed forms, conservation laws, stationary
solutions, exact discrete amplification factors).  Small boxes only, so the
whole file runs in about a minute."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import model as om
from oracle.model import OracleLBM


def make(nx, ny, nz, thermal="D3Q7", q_phase=15, **kw):
    p = W.Params(**kw)
    return OracleLBM(nx, ny, nz, p, q_phase, thermal)


def set_fields(o, phi, u=None, T=None, p=None):
    """Equilibrium state for given fields (the oracle's own init formulas)."""
    shape = (o.nz, o.ny, o.nx)
    phi = np.broadcast_to(phi, shape).astype(float)
    u = np.zeros((3,) + shape) if u is None else np.broadcast_to(u, (3,) + shape).astype(float)
    T = np.zeros(shape) if T is None else np.broadcast_to(T, shape).astype(float)
    p = np.zeros(shape) if p is None else p
    o.h = om.eq_scalar(phi, u, o.Sh)
    o.g = om.eq_hydro(p, u, o.S27)
    if o.lb_thermal:
        o.f = om.eq_scalar(T, u, o.Sf)
    else:
        o.T = T.copy()


# ------------------------------------------------------------ streaming
@pytest.mark.parametrize("walls", [False, True])
def test_pull_moves_populations_along_c(walls):
    o = make(4, 5, 6, walls_z=walls)
    S = o.S27
    src = np.zeros((27, 6, 5, 4))
    x0 = (2, 1, 3)  # (z, y, x)
    for i in range(27):
        src[i][x0] = i + 1.0
    out = o._pull(src, S)
    for i in range(27):
        cx, cy, cz = S.c[i]
        z = x0[0] + cz
        dest = (z % 6, (x0[1] + cy) % 5, (x0[2] + cx) % 4)
        assert out[i][dest] == i + 1.0
    # bounce-back: population leaving z = 0 downward returns reversed in place
    if walls:
        src = np.zeros((27, 6, 5, 4))
        down = [i for i in range(27) if S.c[i, 2] == -1]
        for i in down:
            src[i][0, 2, 1] = 10.0 + i
        out = o._pull(src, S)
        for i in down:
            assert out[S.opp[i]][0, 2, 1] == 10.0 + i
        fo = o._pull(src, S, "abb", 0.25, 0.0)
        for i in down:
            j = S.opp[i]
            assert fo[j][0, 2, 1] == -(10.0 + i) + 2 * S.w[j] * 0.25


# ------------------------------------------------------------ conservation
@pytest.mark.parametrize("walls", [False, True])
def test_phi_mass_conserved(walls):
    w = W.config1()
    p = W.Params(**{**w.params.__dict__, "walls_z": walls, "T_bottom": -0.1, "T_top": 0.2})
    o = OracleLBM(16, 16, 16, p, 15, "D3Q7")
    o.init_droplets([W.Droplet(8.0, 7.5, 8.2, 5.0, 1e-3, -2e-3, 1e-3)])
    m0 = o.macro()["phi"].sum()
    o.step(30)
    m1 = o.macro()["phi"].sum()
    assert abs(m1 - m0) / m0 < 1e-13


def test_uniform_body_force_momentum_growth():
    """Guo forcing: with a uniform force the level-n velocity is (n + 1/2) a
    and the total first moment grows by a per cell per step."""
    g = (1e-5, -2e-5, 3e-5)
    o = make(4, 4, 4, gravity=g)
    set_fields(o, 0.0)
    for n in range(1, 6):
        o.step(1)
        u = o.macro()["u"]
        for a in range(3):
            assert np.abs(u[a] - (n + 0.5) * g[a]).max() < 1e-18
        j = np.einsum("iq,i...->q...", o.S27.c.astype(float), o.g)
        for a in range(3):
            assert abs(j[a].sum() - n * g[a] * 64) < 1e-16


@pytest.mark.parametrize("rho", [1.0, 2.5])
def test_kinetic_energy_of_uniform_flow(rho):
    """The kinetic-energy diagnostic (a10, 1/2 sum rho |u|^2) of a uniform
    flow u = U at density rho over N cells is exactly 1/2 rho |U|^2 N.  A
    droplet is present (phi varies) but sigma = 0 and no gravity, so no force
    acts and u = U in every cell; a missing 1/2, a missing rho or a wrong u
    (e.g. a half-force shift or a lost component) all change the value.  The
    box is periodic: the pulled g of a uniform equilibrium is that
    equilibrium again, so the level's velocity is exactly U."""
    U = (0.012, -0.021, 0.0047)
    nx, ny, nz = 10, 8, 6
    o = make(nx, ny, nz, rho_L=rho, rho_H=rho, sigma_ref=0.0, sigma_T=0.0)
    X = (np.arange(nx) + 0.5)[None, None, :]
    Y = (np.arange(ny) + 0.5)[None, :, None]
    Z = (np.arange(nz) + 0.5)[:, None, None]
    r = np.sqrt((X - nx / 2) ** 2 + (Y - ny / 2) ** 2 + (Z - nz / 2) ** 2)
    phi = 0.5 * (1.0 + np.tanh(2.0 * (2.5 - r) / 2.0))
    set_fields(o, phi, u=np.array(U)[:, None, None, None])
    d = o.diagnostics()
    N = nx * ny * nz
    exact = 0.5 * rho * (U[0] ** 2 + U[1] ** 2 + U[2] ** 2) * N
    assert abs(d["kinetic"] - exact) <= 1e-13 * exact, (d["kinetic"], exact)


@pytest.mark.parametrize("thermal", ["D3Q7", "D3Q19", "RK2", "RK4"])
def test_uniform_heat_source(thermal):
    o = make(4, 3, 5, thermal=thermal)
    set_fields(o, 0.0, T=0.0)
    o.q = np.full((5, 3, 4), 2.5e-3)
    o.step(4)
    T = o.macro()["T"]
    assert np.abs(T - 4 * 2.5e-3).max() < 1e-17


# ------------------------------------------------------------ transport coefficients
def _amp(field, coord, k):
    return 2.0 * np.mean(field * np.sin(k * coord))


def test_shear_wave_viscosity():
    """u_x = U sin(k z) decays as exp(-nu k^2 t), nu = c_s^2 (tau - 1/2)."""
    nu = 0.1
    o = make(1, 1, 32, nu_L=nu, nu_H=nu)
    k = 2 * math.pi / 32
    z = o.Z
    u = np.zeros((3, 32, 1, 1))
    u[0] = 1e-4 * np.sin(k * z)
    set_fields(o, 0.0, u=u)
    o.step(20)
    a0 = _amp(o.macro()["u"][0], z, k)
    o.step(100)
    a1 = _amp(o.macro()["u"][0], z, k)
    rate = -math.log(a1 / a0) / 100
    assert abs(rate / (nu * k * k) - 1) < 0.01


@pytest.mark.parametrize("thermal", ["D3Q7", "D3Q15", "D3Q19", "D3Q27"])
def test_lb_heat_diffusion_rate(thermal):
    alpha = 0.05
    o = make(32, 1, 1, thermal=thermal, alpha_L=alpha, alpha_H=alpha)
    k = 2 * math.pi / 32
    x = o.X
    set_fields(o, 0.0, T=1e-2 * np.sin(k * x))
    o.step(10)
    a0 = _amp(o.macro()["T"], x, k)
    o.step(200)
    a1 = _amp(o.macro()["T"], x, k)
    rate = -math.log(a1 / a0) / 200
    assert abs(rate / (alpha * k * k) - 1) < 0.01


@pytest.mark.parametrize("scheme", ["RK2", "RK4"])
def test_rk_amplification_exact(scheme):
    """RK on the 7-point Laplacian: T^{n+1} = P(z) T^n with z = alpha(2cos k - 2),
    P = 1 + z + z^2/2 (RK2, midpoint) or the quartic Taylor polynomial (RK4)."""
    alpha = 0.1
    o = make(16, 1, 1, thermal=scheme, alpha_L=alpha, alpha_H=alpha)
    k = 2 * math.pi * 3 / 16
    T0 = 0.3 * np.sin(k * o.X)
    set_fields(o, 0.0, T=T0)
    z = alpha * (2 * math.cos(k) - 2)
    P = 1 + z + z * z / 2 + ((z ** 3 / 6 + z ** 4 / 24) if scheme == "RK4" else 0)
    o.step(5)
    assert np.abs(o.T - P ** 5 * T0).max() < 1e-15


@pytest.mark.parametrize("thermal", ["D3Q7", "D3Q27", "RK2", "RK4"])
def test_wall_conduction_linear_profile_exact(thermal):
    """Between walls at T_b, T_t the conduction profile is linear in the
    wall-normal coordinate with the walls half a cell outside the first and
    last cell; anti-bounce-back (LB) and the ghost 2T_w - T (RK) keep it exactly."""
    o = make(2, 2, 12, thermal=thermal, walls_z=True, T_bottom=-0.5, T_top=0.5)
    o.init_droplets([])
    T_lin = -0.5 + o.Z / 12.0
    o.step(40)
    assert np.abs(o.macro()["T"] - T_lin).max() < 1e-14


# ------------------------------------------------------------ interface
def _slab(z, z1, z2, xi):
    return 0.5 * (np.tanh(2 * (z - z1) / xi) - np.tanh(2 * (z - z2) / xi))


def test_tanh_profile_is_stationary():
    """phi = 1/2 (1 + tanh(2 x / xi)) solves the conservative Allen-Cahn
    equation at rest; a wrong source scale changes the width by a factor 3.
    On the lattice the stationary profile differs from the continuous tanh by
    O(1/xi^2) (width +0.9%, 4e-3 at xi = 5); it must be stationary."""
    from scipy.optimize import curve_fit
    xi = 5.0
    o = make(1, 1, 64, xi=xi, sigma_T=0.0, mobility=0.02)
    z = o.Z
    phi0 = _slab(z, 16.0, 48.0, xi)
    set_fields(o, phi0)
    o.step(1000)
    phi_a = o.macro()["phi"]
    o.step(1000)
    phi = o.macro()["phi"]
    assert np.abs(phi - phi_a).max() < 2e-4
    assert np.abs(phi - phi0).max() < 5e-3
    zz = z[:, 0, 0]
    popt, _ = curve_fit(lambda zz, a, b, w: _slab(zz, a, b, w), zz, phi[:, 0, 0],
                        p0=(15.0, 47.0, 4.0))
    assert abs(popt[2] / xi - 1) < 0.02
    assert abs(popt[0] - 16.0) < 0.05 and abs(popt[1] - 48.0) < 0.05


def test_planar_interface_advected_with_flow():
    """A uniform velocity carries a planar interface: after N steps the
    profile is the initial one shifted by U N (Galilean invariance of the
    phase-field equation, Eq. phasefield)."""
    from scipy.optimize import curve_fit
    xi, U = 5.0, 0.02
    o = make(1, 1, 64, xi=xi, sigma_T=0.0)
    z = o.Z
    u = np.zeros((3, 64, 1, 1))
    u[2] = U
    set_fields(o, _slab(z, 16.0, 40.0, xi), u=u)
    o.step(300)
    phi = o.macro()["phi"][:, 0, 0]
    popt, _ = curve_fit(lambda zz, a, b: _slab(zz, a, b, xi), z[:, 0, 0], phi, p0=(20.0, 44.0))
    shift = U * 300.5   # the level-300 fields follow 300 collisions + 1 streaming
    assert abs(popt[0] - 16.0 - shift) < 0.1 and abs(popt[1] - 40.0 - shift) < 0.1


def test_laplace_pressure_cylinder():
    """Static cylinder: Delta p = sigma / R (Young-Laplace in 2D), with
    p = rho c_s^2 p* (p* the zeroth moment of g, Sec. 2.2)."""
    R, sigma, xi = 8.0, 5e-3, 5.0
    o = make(32, 32, 1, sigma_ref=sigma, sigma_T=0.0, xi=xi, nu_L=0.1, nu_H=0.1,
             mobility=0.02)
    r = np.sqrt((o.X - 16.0) ** 2 + (o.Y - 16.0) ** 2)
    set_fields(o, 0.5 * (1 + np.tanh(2 * (R - r) / xi)))
    o.step(1000)
    m = o.macro()
    pin = m["p"][r < 3].mean()
    pout = m["p"][r > 14].mean()
    dp = (pin - pout) / 3.0
    assert abs(dp / (sigma / R) - 1) < 0.05


def test_marangoni_shear_between_walls():
    """Planar interface between no-slip walls under a tangential gradient G.
    The Marangoni part of Eq. F_s, f_x = (3/2) xi sigma_T |d phi/dz|^2 G
    (integral sigma_T G across the interface), drives the steady Stokes flow
    mu u'' = -f_x with u = 0 on the half-way walls; compare with that exact
    solution (Green's-function quadrature on the continuous tanh profile)."""
    H, nu, G, sT, xi = 32, 0.5, 1e-2, -5e-4, 5.0
    o = make(1, 1, H, nu_L=nu, nu_H=nu, sigma_T=sT, grad_T=(G, 0.0, 0.0),
             walls_z=True, alpha_L=0.05, alpha_H=0.05, xi=xi)
    zi = H / 2
    set_fields(o, 0.5 * (1 + np.tanh(2 * (o.Z - zi) / xi)))
    o.step(1500)
    ux = o.macro()["u"][0][:, 0, 0]
    lo, hi = 0.0, float(H)
    s = np.linspace(lo, hi, 200001)
    dphi = (1.0 / xi) / np.cosh(2 * (s - zi) / xi) ** 2
    f = 1.5 * xi * sT * G * dphi ** 2
    z = np.arange(H, dtype=float) + 0.5
    exact = np.empty(H)
    for j, zz in enumerate(z):
        gr = np.where(zz <= s, (zz - lo) * (hi - s), (s - lo) * (hi - zz)) / (hi - lo)
        exact[j] = np.trapezoid(gr * f, s) / nu
    ui_sharp = sT * G / (nu * (2.0 / (H / 2)))
    assert abs(np.trapezoid(f, s) / (sT * G) - 1) < 1e-6
    # On the lattice the force integral falls short of sigma_T G by O(1/xi^2)
    # (the central difference underestimates the tanh slope: 0.95 at xi = 5).
    ratio = o.macro()["F"][0].sum() / (sT * G)
    assert 0.93 < ratio < 1.0
    # the flow is the Stokes response to that force
    assert np.abs(ux - ratio * exact).max() < 0.015 * abs(ui_sharp)


def test_centred_droplet_does_not_move():
    o = make(16, 16, 16, sigma_T=-5e-4, grad_T=(0.0, 0.0, 0.0))
    # the box centre: the lattice is mirror-symmetric about it
    o.init_droplets([W.Droplet(8.0, 8.0, 8.0, 5.0)])
    c0 = np.array(o.diagnostics()["centroid"])
    o.step(40)
    c1 = np.array(o.diagnostics()["centroid"])
    assert np.abs(c1 - c0).max() < 1e-12


def test_mobility_sets_interface_relaxation_rate():
    """A tanh profile of width xi' != xi relaxes at the rate given by the
    conservative Allen-Cahn flux J = M (grad phi - 4 phi (1-phi)/xi n):
    d phi/dt = M (1/xi' - 1/xi) 4 (1 - 2 phi) phi'  (Eq. phasefield), which
    fixes the relaxation rate omega_phi = 1/(1/2 + M/c_s^2)."""
    M, xi, xip = 0.02, 5.0, 10.0
    o = make(1, 1, 96, xi=xi, mobility=M, sigma_ref=0.0, sigma_T=0.0)
    z = o.Z[:, 0, 0]
    set_fields(o, _slab(o.Z, 24.0, 72.0, xip))
    o.step(10)
    p0 = o.macro()["phi"][:, 0, 0]
    o.step(10)
    p1 = o.macro()["phi"][:, 0, 0]
    rate = (p1 - p0) / 10.0
    ph = _slab(z, 24.0, 72.0, xip)           # profile at the midpoint, to O(dt)
    sgn = np.where(z < 48, 1.0, -1.0)        # n points into the slab
    dph = sgn * 4 * ph * (1 - ph) / xip
    want = M * (1 / xip - 1 / xi) * 4 * (1 - 2 * ph) * dph * sgn
    assert np.abs(rate - want).max() < 0.05 * np.abs(want).max()


def test_heat_source_integral_and_cutoff():
    """Eq. HeatSource: sum over the lattice of Q exp(-2 r^2/w^2) equals the
    Gaussian integral Q (pi w^2/2)^(3/2) (w = 6 >> 1); with the cut-off
    r <= d (read: the printed >= would heat everything but the spot) the
    total is Q (pi w^2/2)^(3/2) [erf(s) - 2 s exp(-s^2)/sqrt(pi)], s = sqrt2 d/w."""
    from math import erf, exp, pi, sqrt
    Q, w = 0.2, 6.0
    o = OracleLBM(48, 48, 48, W.Params(), 15, "D3Q7",
                  sources=[W.HeatSource(24.0, 24.3, 23.6, Q, w)])
    full = Q * (pi * w * w / 2) ** 1.5
    assert abs(o.q.sum() / full - 1) < 1e-9
    d = 8.0
    o2 = OracleLBM(48, 48, 48, W.Params(), 15, "D3Q7",
                   sources=[W.HeatSource(24.5, 24.5, 24.5, Q, w, d)])
    s = sqrt(2) * d / w
    cut = full * (erf(s) - 2 * s * exp(-s * s) / sqrt(pi))
    # lattice sum of a truncated Gaussian: discretisation of the sharp edge
    assert abs(o2.q.sum() / cut - 1) < 0.01
    assert o2.q[24, 24, 24] == Q


def test_heat_field_layout_matches_sources_and_patches():
    """A per-cell heat field laid out [z][y][x] (x fastest) is the same q_T
    as the Gaussian source and the heater patch it samples, on a box whose
    three sides differ (a transposed layout puts the heat elsewhere)."""
    nx, ny, nz = 7, 5, 4
    src = W.HeatSource(2.3, 3.1, 1.6, 0.01, 1.5)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                          indexing="ij")
    gauss = src.Q * np.exp(-2.0 * ((x - src.x) ** 2 + (y - src.y) ** 2 + (z - src.z) ** 2)
                           / src.w ** 2)
    a = OracleLBM(nx, ny, nz, W.Params(), 15, "D3Q7", sources=[src])
    b = OracleLBM(nx, ny, nz, W.Params(), 15, "D3Q7")
    b.add_heat_field(gauss.ravel())
    assert np.allclose(a.q, b.q, rtol=1e-14, atol=0) and a.q.max() > 0
    patches = W.HeaterPatches(z=1, sx=2, sy=3, x0=[4], y0=[1], intensity=[0.02])
    c = OracleLBM(nx, ny, nz, W.Params(), 15, "D3Q7", patches=patches)
    box = np.zeros(nx * ny * nz)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if k == 1 and 1 <= j < 4 and 4 <= i < 6:
                    box[(k * ny + j) * nx + i] = 0.02
    e = OracleLBM(nx, ny, nz, W.Params(), 15, "D3Q7")
    e.add_heat_field(box)
    assert np.array_equal(c.q, e.q)


@pytest.mark.parametrize("thermal", ["D3Q7", "D3Q19", "RK2", "RK4"])
def test_heat_field_total_heat_grows_by_its_sum(thermal):
    """Periodic box at rest: streaming and the periodic difference operators
    conserve sum T, so n steps with a heat field q add exactly n * sum q."""
    o = make(6, 5, 4, thermal=thermal)
    set_fields(o, 0.0, T=0.0)
    q = W.heater_field(9, (4, 5, 6))
    o.add_heat_field(q)
    o.step(5)
    T = o.macro()["T"]
    assert abs(T.sum() / (5 * q.sum()) - 1) < 1e-12
    assert np.abs(T).max() < 5 * q.max()        # diffusion spread the spots


@pytest.mark.parametrize("thermal,tol", [("D3Q7", 4e-3), ("RK4", 3e-2)])
def test_two_layer_conduction_steady_state(thermal, tol):
    """Conductivity ratio 1/5 across a planar diffuse interface between two
    walls (T = 1 below, 0 above), no flow.  The steady state of
    dT/dt = div(alpha(phi) grad T) carries a constant flux, so
    T(z) = 1 - int_0^z dz'/alpha / int_0^H dz'/alpha (quadrature of the
    tanh profile's alpha).  The LB (conservative by construction) and the RK
    finite differences (alpha lap T + grad alpha . grad T) must reach it to
    their discretisation error; a dropped or sign-flipped grad alpha . grad T
    term moves the interface temperature by more than 0.3."""
    from scipy.integrate import quad
    nz, xi, aL, aH, zc = 16, 3.0, 0.5, 0.1, 8.0
    o = make(1, 1, nz, thermal=thermal, alpha_L=aL, alpha_H=aH, xi=xi, sigma_ref=1e-4,
             sigma_T=0.0, walls_z=True, T_bottom=1.0, T_top=0.0)
    phi = 0.5 * (1 + np.tanh(2 * (o.Z - zc) / xi))
    set_fields(o, phi, T=1.0 - o.Z / nz)
    o.step(1200)
    T = o.macro()["T"][:, 0, 0]

    def inv_alpha(z):
        return 1.0 / (aL + 0.5 * (1 + math.tanh(2 * (z - zc) / xi)) * (aH - aL))

    total = quad(inv_alpha, 0, nz, points=[zc])[0]
    exact = np.array([1 - quad(inv_alpha, 0, z, points=[zc] if z > zc else None)[0] / total
                      for z in o.Z[:, 0, 0]])
    assert np.abs(T - exact).max() < tol
    assert np.abs(o.macro()["u"]).max() < 1e-6


@pytest.mark.parametrize("thermal,tol", [("D3Q7", 0.05), ("RK4", 0.03)])
def test_modulated_wall_conduction_closed_form(thermal, tol):
    """Bottom wall T_h + T_0 cos(omega x) (the heated channel's wall,
    Sec. 3.1), top wall T_c, no flow: the steady state solves Laplace's
    equation, T = T_h + (T_c - T_h) z / H + T_0 cos(omega x) sinh(omega (H - z))
    / sinh(omega H), walls on the faces z = 0 and z = H, x at cell centres.
    Second order in omega (the error falls 3.6x when omega halves); a
    half-cell shift of x or a flipped amplitude is off by 0.4 or more."""
    nx, nz = 32, 16
    o = make(nx, 1, nz, thermal=thermal, alpha_L=0.2, alpha_H=0.2, sigma_T=0.0, walls_z=True,
             T_bottom=20.0, T_top=10.0, T_bottom_amp=4.0, T_bottom_waves=1)
    set_fields(o, 0.0, T=20.0 - 10.0 * o.Z / nz)
    o.step(800)
    w = 2 * math.pi / nx
    exact = (20.0 - 10.0 * o.Z / nz
             + 4.0 * np.cos(w * o.X) * np.sinh(w * (nz - o.Z)) / np.sinh(w * nz))
    assert np.abs(o.macro()["T"] - exact).max() < tol


@pytest.mark.parametrize("thermal", ["D3Q7", "D3Q19", "RK4"])
def test_heat_capacity_sets_diffusivity(thermal):
    """Uniform rho = 2, c_p = 1.5 and kappa = 0.15 (Eq. temperature): the
    diffusivity is kappa / (rho c_p) = 0.05, so a sine mode decays at
    0.05 k^2 per step (LB, to 1 %) or by the exact RK4 amplification factor
    of the 7-point Laplacian at that diffusivity; taking kappa itself as the
    diffusivity would triple the rate."""
    kap, rho, cp = 0.15, 2.0, 1.5
    alpha = kap / (rho * cp)
    o = make(32, 1, 1, thermal=thermal, alpha_L=kap, alpha_H=kap, rho_L=rho, rho_H=rho, cp_L=cp, cp_H=cp)
    k = 2 * math.pi / 32
    x = o.X
    T0 = 1e-2 * np.sin(k * x)
    set_fields(o, 0.0, T=T0)
    if thermal == "RK4":
        z = alpha * (2 * math.cos(k) - 2)
        P = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
        o.step(5)
        assert np.abs(o.T - P ** 5 * T0).max() < 1e-15
        return
    o.step(10)
    a0 = _amp(o.macro()["T"], x, k)
    o.step(200)
    a1 = _amp(o.macro()["T"], x, k)
    rate = -math.log(a1 / a0) / 200
    assert abs(rate / (alpha * k * k) - 1) < 0.01


def _heat_capacity_steady_profile(nz, zc, xi, kL, kH, CL_of, q):
    """Steady state of C dT/dt = d/dz (kappa dT/dz) + C q between walls at
    T = 0 (faces z = 0 and z = nz), kappa and C functions of the tanh profile
    phi(z): kappa T' = A - q F(z), F = int_0^z C, and T(nz) = 0 fixes A.
    Also returns the profile of the model that drops the heat-capacity
    gradient term, (alpha T')' = -q with alpha = kappa / C."""
    from scipy.integrate import quad

    def phi(z):
        return 0.5 * (1 + math.tanh(2 * (z - zc) / xi))

    def kap(z):
        return kL + phi(z) * (kH - kL)

    def C(z):
        return CL_of(phi(z))

    def F(z):
        return quad(C, 0, z, points=[zc] if z > zc else None)[0]

    def integ(fun, z):
        return quad(fun, 0, z, points=[zc] if z > zc else None, limit=200)[0]

    A = q * integ(lambda s: F(s) / kap(s), nz) / integ(lambda s: 1 / kap(s), nz)
    B = q * integ(lambda s: s * C(s) / kap(s), nz) / integ(lambda s: C(s) / kap(s), nz)
    zs = np.arange(nz) + 0.5
    exact = np.array([integ(lambda s: (A - q * F(s)) / kap(s), z) for z in zs])
    wrong = np.array([integ(lambda s: (B - q * s) * C(s) / kap(s), z) for z in zs])
    return exact, wrong


def _steady_heating_error(thermal, kw, scale=1):
    nz, xi, zc, q = 16 * scale, 3.0 * scale, 8.0 * scale, 1e-3 / scale ** 2
    kL, kH = 0.5, 0.25
    o = make(1, 1, nz, thermal=thermal, alpha_L=kL, alpha_H=kH, xi=xi, sigma_ref=1e-4,
             sigma_T=0.0, walls_z=True, T_bottom=0.0, T_top=0.0, **kw)
    exact, wrong = _heat_capacity_steady_profile(nz, zc, xi, kL, kH, lambda ph: 1.0 + 2.0 * ph, q)
    phi = 0.5 * (1 + np.tanh(2 * (o.Z - zc) / xi))
    set_fields(o, phi, T=exact.reshape(nz, 1, 1))
    o.add_heat_field(np.full(nz, q))
    o.step(1500 * scale * scale)
    T = o.macro()["T"][:, 0, 0]
    peak = np.abs(exact).max()
    assert np.abs(o.macro()["u"]).max() < 1e-6
    return np.abs(T - exact).max() / peak, np.abs(wrong - exact).max() / peak


@pytest.mark.parametrize("thermal,tol", [("D3Q7", 4e-2), ("D3Q27", 4e-2), ("RK4", 2e-2)])
@pytest.mark.parametrize("ratio", ["cp", "rho"])
def test_heat_capacity_ratio_steady_heating(thermal, tol, ratio):
    """A planar diffuse interface (xi = 3) between walls at T = 0 sixteen
    cells apart, uniform heating q of dT/dt, conductivity ratio 1/2 and a
    heat-capacity ratio 3 carried by c_p (or by the density, Eq. rho(phi),
    with c_p = 1): the steady state of Eq. temperature solves
    (kappa T')' = -q rho c_p (closed form by quadrature).  The solvers reach
    it to their discretisation error (measured 2.7 % of the peak for the
    LB, 1.4 % for RK4, second order: see the next test); the model without
    the grad(rho c_p) term of the LB source is off by 27 %."""
    err, gap = _steady_heating_error(thermal, dict(cp_L=1.0, cp_H=3.0) if ratio == "cp"
                                     else dict(rho_L=1.0, rho_H=3.0))
    print(thermal, ratio, "steady error", err, "wrong model", gap)
    assert gap > 0.25
    assert err < tol


def test_heat_capacity_steady_heating_second_order():
    """The same problem at twice the resolution (interface width, distance
    and heating scaled): the LB error falls by about 4."""
    e1, _ = _steady_heating_error("D3Q7", dict(cp_L=1.0, cp_H=3.0))
    e2, _ = _steady_heating_error("D3Q7", dict(cp_L=1.0, cp_H=3.0), scale=2)
    print("steady heating error", e1, e2, e1 / e2)
    assert 3.3 < e1 / e2 < 4.8


def test_conductivity_ratio_lb_conserves_heat():
    """Periodic box at rest, alpha_H = alpha_L / 5 with a droplet-shaped phi:
    the per-cell relaxation rate leaves sum T unchanged (no sources)."""
    o = make(8, 6, 5, thermal="D3Q15", alpha_L=0.2, alpha_H=0.04, sigma_T=0.0)
    z, y, x = o.Z, o.Y, o.X
    phi = 0.5 * (1 + np.tanh(2 * (2.5 - np.sqrt((x - 4) ** 2 + (y - 3) ** 2 + (z - 2.5) ** 2)) / 2.0))
    T = W.random_state(4, (5, 6, 8), 0.1)
    set_fields(o, phi, T=T)
    s0 = o.macro()["T"].sum()
    o.step(6)
    assert abs(o.macro()["T"].sum() - s0) < 1e-13 * np.abs(T).sum()


@pytest.mark.parametrize("thermal", ["D3Q7", "RK2", "RK4"])
def test_background_gradient_advection_source(thermal):
    """T_total = T + G.(x - x0): a uniform flow U across the imposed gradient
    changes T at the rate -U.G (Eq. temperature, advection term)."""
    U, G = 2e-3, 3e-3
    o = make(4, 4, 4, thermal=thermal, grad_T=(G, 0.0, 0.0))
    u = np.zeros((3, 4, 4, 4))
    u[0] = U
    set_fields(o, 0.0, u=u)
    o.step(6)
    T = o.macro()["T"]
    assert np.abs(T + 6 * U * G).max() < 1e-15


@pytest.mark.parametrize("scheme", ["RK2", "RK4"])
def test_rk_advection_diffusion_amplification(scheme):
    """Uniform u: the central-difference / 7-point operator has symbol
    z = -i U sin k + alpha (2 cos k - 2); T^n = Im(P(z)^n e^{ikx}) exactly."""
    U, alpha = 0.05, 0.08
    o = make(16, 1, 1, thermal=scheme, alpha_L=alpha, alpha_H=alpha)
    k = 2 * math.pi * 2 / 16
    u = np.zeros((3, 1, 1, 16))
    u[0] = U
    set_fields(o, 0.0, u=u, T=np.sin(k * o.X))
    z = -1j * U * math.sin(k) + alpha * (2 * math.cos(k) - 2)
    P = 1 + z + z * z / 2 + ((z ** 3 / 6 + z ** 4 / 24) if scheme == "RK4" else 0)
    o.step(4)
    want = np.imag(P ** 4 * np.exp(1j * k * o.X))
    assert np.abs(o.T - want).max() < 1e-14


def test_wall_ghost_gives_exact_temperature_gradient():
    o = make(2, 2, 10, walls_z=True, T_bottom=-0.3, T_top=0.7)
    o.init_droplets([])
    gT = o.macro()["gT"]
    assert np.abs(gT[2] - 1.0 / 10).max() < 1e-15
    assert np.abs(gT[0]).max() < 1e-16 and np.abs(gT[1]).max() < 1e-16


def test_initial_droplet_profile_properties():
    """Initial phi: 1/2 exactly at distance R from the centre, tanh profile
    (Sec. 3.1 initialisation), periodic minimum-image distances."""
    p = W.Params()
    o = OracleLBM(32, 32, 32, p, 15, "D3Q7")
    # cell k is centred at k + 1/2
    o.init_droplets([W.Droplet(16.5, 16.5, 16.5, 8.0), W.Droplet(1.0, 5.0, 16.0, 5.0)])
    phi = o.h.sum(axis=0)
    assert abs(phi[16, 16, 24] - 0.5) < 1e-15 and abs(phi[16, 24, 16] - 0.5) < 1e-15
    assert phi[16, 16, 16] > 0.99
    # second droplet wraps around x = 0: cells 1 + j and -j mirror about x = 1
    for j in range(0, 5):
        assert phi[16, 5, (1 + j) % 32] == phi[16, 5, (-j) % 32]
    assert phi[16, 5, 31] > 0.9


# ------------------------------------------------------------ density ratio
def test_density_ratio_laplace_cylinder():
    """Static cylinder at density ratio rho_H / rho_L = 10 (F_p and F_mu of
    Sec. 2.2 active): the pressure p = rho c_s^2 p* jumps by sigma / R across
    the interface (Young-Laplace in 2D) within 5 %."""
    R, sigma, xi = 8.0, 1e-2, 4.0
    o = make(32, 32, 1, sigma_ref=sigma, sigma_T=0.0, xi=xi, nu_L=0.1, nu_H=0.1,
             mobility=0.02, rho_L=1.0, rho_H=10.0)
    r = np.sqrt((o.X - 16.0) ** 2 + (o.Y - 16.0) ** 2)
    set_fields(o, 0.5 * (1 + np.tanh(2 * (R - r) / xi)))
    o.step(1000)
    m = o.macro()
    pr = m["p"] * m["rho"] / 3.0
    dp = pr[r < 3].mean() - pr[r > 14].mean()
    assert abs(dp / (sigma / R) - 1) < 0.05, dp / (sigma / R)
    assert np.abs(m["u"]).max() < 1e-4          # spurious currents stay small


def _layered_channel_closed_form(H, xi, rho_L, rho_H, nu, g, z, n=400001):
    """Steady two-layer channel flow under a body force rho(z) g along x, no
    slip at z = 0 and z = H: d/dz (mu u') = -rho g with mu = rho nu(tau(phi))
    and rho linear in the equilibrium phase-field profile (heavy phase below
    z = H/2), integrated by quadrature (trapezoid rule on a fine grid):
    mu u' = -g int_0^z rho + C, u = int_0^z (mu u') / mu, C from u(H) = 0."""
    zz = np.linspace(0.0, H, n)
    ph = 0.5 * (1 + np.tanh(2 * (H / 2 - zz) / xi))
    rho = rho_L + ph * (rho_H - rho_L)
    mu = rho * nu
    dz = zz[1] - zz[0]

    def cum(f):
        return np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * dz)])
    I1 = cum(-g * cum(rho) / mu)
    I2 = cum(1.0 / mu)
    u = I1 - I1[-1] / I2[-1] * I2
    return np.interp(z, zz, u)


def test_density_ratio_layered_channel_second_order():
    """Two layers (rho_H / rho_L = 10, equal kinematic viscosity, so a
    dynamic-viscosity ratio of 10) between no-slip walls, driven by gravity
    along x: the steady velocity converges at second order to the closed form
    of d/dz (mu u') = -rho g for the same diffuse interface.  The viscous
    correction F_mu (strain from the non-equilibrium moments of g) is what
    makes the lattice solve this equation: without it the error does not
    fall with resolution."""
    errs = []
    for H, xi, steps in ((16, 3.0, 1500), (32, 6.0, 4000)):
        nu, g = 0.3, 1e-6
        o = make(1, 1, H, rho_L=1.0, rho_H=10.0, nu_L=nu, nu_H=nu, sigma_ref=1e-3,
                 sigma_T=0.0, xi=xi, mobility=0.02, walls_z=True, gravity=(g, 0.0, 0.0))
        set_fields(o, 0.5 * (1 + np.tanh(2 * (H / 2 - o.Z) / xi)))
        o.step(steps)
        u = o.macro()["u"][0][:, 0, 0]
        ref = _layered_channel_closed_form(H, xi, 1.0, 10.0, nu, g, o.Z[:, 0, 0])
        errs.append(float(np.sqrt(((u - ref) ** 2).sum() / (ref ** 2).sum())))
    assert errs[0] < 0.03 and errs[1] < 0.008, errs
    assert errs[0] / errs[1] > 3.5, errs           # second order in the lattice spacing


# ------------------------------------------------------------ moving walls, wetting
def test_couette_flow_moving_top_wall_exact():
    """Top wall moving at U along x, bottom wall at rest (the sheared channel
    of Sec. 3.3): the steady velocity is the linear Couette profile
    u_x = U z / H at the cell centres, which half-way bounce-back with the
    moving-wall term reproduces to round-off."""
    H, U = 16, 0.01
    o = make(1, 1, H, walls_z=True, nu_L=0.3, nu_H=0.3, sigma_ref=0.0, sigma_T=0.0,
             wall_u_top=(U, 0.0))
    set_fields(o, 0.0)
    o.step(2000)
    u = o.macro()["u"]
    assert np.abs(u[0][:, 0, 0] - U * o.Z[:, 0, 0] / H).max() < 1e-9 * U
    assert np.abs(u[1]).max() < 1e-15 and np.abs(u[2]).max() < 1e-15


def test_moving_walls_conserve_phi_mass_and_heat_balance():
    """Both walls moving tangentially (in x and y), a droplet touching the
    top wall region: phi mass is conserved to round-off (the moving-wall
    terms of the h populations cancel in pairs), and at rest in a uniform
    temperature T_w = T_wall the thermal anti-bounce-back with the moving
    wall keeps T uniform."""
    o = make(12, 8, 10, walls_z=True, wall_u_top=(0.02, -0.01), wall_u_bottom=(-0.01, 0.005),
             T_bottom=0.3, T_top=0.3, sigma_T=0.0)
    o.init_droplets([W.Droplet(6.0, 4.0, 7.0, 3.0)])
    m0 = o.macro()["phi"].sum()
    o.step(60)
    m = o.macro()
    assert abs(m["phi"].sum() - m0) / m0 < 1e-13
    assert np.abs(m["T"] - 0.3).max() < 1e-3      # u is small; T stays near the wall value


def _tilted_interface_angle(theta_bc_bottom, theta_bc_top, steps, nx=40, nz=20, theta=60.0, xi=4.0):
    """A slab of phi = 1 bounded on the right by a plane tilted at theta to
    the walls (so the heavy phase meets the bottom wall at 180 - theta and
    the top wall at theta); returns the tilt of that interface (from the phi
    = 1/2 crossings of the rows next to the walls) after the given steps."""
    o = make(nx, 1, nz, walls_z=True, sigma_ref=5e-3, sigma_T=0.0, xi=xi, mobility=0.05,
             nu_L=0.1, nu_H=0.1, theta_bottom=theta_bc_bottom, theta_top=theta_bc_top)
    ct = 1.0 / math.tan(math.radians(theta))
    s = math.sin(math.radians(theta))
    right = (o.X - (nx / 2 + (o.Z - nz / 2) * ct)) * s
    left = (o.X - (nx / 2 - 10 + (o.Z - nz / 2) * ct)) * s
    set_fields(o, np.minimum(0.5 * (1 + np.tanh(-2 * right / xi)), 0.5 * (1 + np.tanh(2 * left / xi))))
    o.step(steps)
    ph = o.macro()["phi"][:, 0, :]
    xs = []
    for k in (2, nz - 3):
        row = ph[k]
        i = np.where((row[:-1] >= 0.5) & (row[1:] < 0.5))[0][-1]
        xs.append(i + 0.5 + (row[i] - 0.5) / (row[i] - row[i + 1]))
    return math.degrees(math.atan2(nz - 5, xs[1] - xs[0]))


def test_wetting_condition_holds_the_contact_angle():
    """Contact angle (the wetting condition of the conservative phase field,
    Sec. 3.3 reading): a planar interface meeting the walls at the angles the
    walls prescribe (120 / 60 degrees through phi = 1) keeps its tilt of 60
    degrees within 4 degrees over 1000 steps, while with neutral walls (90
    degrees, the mirror ghost) it turns towards the vertical by more than
    5 degrees; a wrong sign of the condition would turn it further still."""
    wet = _tilted_interface_angle(120.0, 60.0, 1000)
    neutral = _tilted_interface_angle(90.0, 90.0, 1000)
    assert abs(wet - 60.0) < 4.0, wet
    assert neutral - 60.0 > 5.0, neutral
    assert neutral > wet


def test_wetting_ghost_formula_properties():
    """The ghost value of the wetting condition: g = a at 90 degrees; at
    other angles (a - g) = -k w (1 - w) with w = (a + g) / 2 to round-off;
    g > a (phi = 1 drawn to the wall) for angles below 90 degrees."""
    o = make(4, 4, 4, walls_z=True, xi=4.0)
    a = np.linspace(0.0, 1.0, 11)
    assert np.array_equal(o._wet_ghost(a, 90.0), a)
    for th in (30.0, 60.0, 120.0, 150.0):
        g = o._wet_ghost(a, th)
        k = 4.0 / 4.0 * math.cos(math.radians(th))
        w = 0.5 * (a + g)
        assert np.abs((a - g) + k * w * (1 - w)).max() < 1e-15
        inner = (a > 0) & (a < 1)
        assert np.all((g[inner] > a[inner]) == (th < 90.0))
