"""Whole-lattice FP64 oracle of one thermocapillary phase-field LBM time step.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every array is
float64; PDF arrays are shaped (Q, nz, ny, nx), scalar fields (nz, ny, nx),
vector fields (3, nz, ny, nx); x is the fastest axis.

Time stepping (Sec. 4.1, Alg. 1 and Alg. 2; pull "one step, two
grid" scheme): the stored PDFs are post-collision values.  One step

  a1  pulls every PDF, p*_i(x) = p_i(x - c_i)   (half-way bounce-back for
      h, g and anti-bounce-back for f at z walls),
  a2  takes the zeroth moments phi = sum h*, p* = sum g*, T = sum f*,
  a3  forms grad phi, lap phi, grad T with the isotropic D3Q27 operators,
  a4  forms n, F^phi, sigma(T), mu_phi,
  a5  forms F = F_s + F_b (+ F_p),
  a6  forms u = sum c_i g*_i + F/(2 rho),
  a7  collides h (single rate, Guo source),
  a8  collides g in central-moment space (Guo forcing in moment space),
  a9  collides f (single rate, + w_i q_T)   or a9' advances T by RK2/RK4,
and all macroscopic quantities used in the collisions are those computed
from the pulled PDFs of this step.  The first step pulls the initial
equilibrium PDFs.

Readings of passages that the paper leaves open or prints garbled (the CUDA
path implements the same readings):
  * relaxation rates of Eq. pflbm-tau / thlbm-tau are read as rates with the
    diffusivity divided by c_s^2: omega = 1 / (1/2 + M / c_s^2);
  * nu = c_s^2 (tau - 1/2) (the paper prints nu = tau c_s^2);
  * the interface force of Eq. phasefieldforce enters as the Guo source
    S_i = (1 - omega_phi/2) w_i (c_i . F^phi), whose first moment
    c_s^2 (1 - omega_phi/2) F^phi recovers the flux M 4 phi (1-phi)/xi n;
  * |grad phi^2| in F_s is read as |grad phi|^2;
  * the chemical potential (not printed) is the double-well form
    mu_phi = 4 beta phi (phi - 1)(phi - 1/2) - kappa lap phi,
    beta = 12 sigma / xi, kappa = 3 sigma xi / 2, with the local sigma(T);
  * Guo forcing "in collision space" for g: the force's central moments are
    those of S_i = w_i [(c_i - u)/c_s^2 + (c_i . u) c_i / c_s^4] . a,
    a = F / rho; second-order central moments relax with 1/tau(phi), all
    moments of order >= 3 with ``omega_high`` (1 by default);
  * walls: half-way bounce-back (h, g), anti-bounce-back f_i = -f_opp +
    2 w_i T_w (f), mirror ghost for phi (neutral wetting), ghost
    T_g = 2 T_w - T for temperature stencils;
  * heat source Eq. HeatSource is non-zero for r^2 <= d_s^2 (printed >=);
  * RK2 (Eq. rk2) is the midpoint rule T + R(T + K1/2);
  * the imposed background gradient G enters as T_total = T + G.(x - x_0);
    the evolved T is the periodic remainder, with source -u.G.
"""
from __future__ import annotations

import itertools
import math
from math import comb
from typing import Dict, Iterable, Optional, Sequence

import numpy as np

from .stencils import stencil

CS2 = 1.0 / 3.0

# Central-moment exponents (a, b, c) in {0,1,2}^3 for the D3Q27 moment space.
MOMENT_EXPONENTS = np.array(list(itertools.product(range(3), repeat=3)),
                            dtype=np.int64)


def raw_moment_matrix(c: np.ndarray) -> np.ndarray:
    """M[k, i] = c_ix^a c_iy^b c_iz^c for the exponents (a, b, c) of moment k."""
    E = MOMENT_EXPONENTS
    M = np.ones((len(E), len(c)))
    for k, e in enumerate(E):
        for i, ci in enumerate(c):
            M[k, i] = float(ci[0] ** e[0] * ci[1] ** e[1] * ci[2] ** e[2])
    return M


def central_moments(pdf: np.ndarray, u: np.ndarray, c: np.ndarray) -> np.ndarray:
    """kappa_abc = sum_i pdf_i (c_ix-u_x)^a (c_iy-u_y)^b (c_iz-u_z)^c, by definition.

    (Central moments in the sense of the cascaded/central-moment LBM the
    paper builds on, Sec. 2.2.)  The sum over i runs as one array reduction."""
    shp = (len(c),) + (1,) * (pdf.ndim - 1)
    # powers[a][e][i] = (c_ia - u_a)^e, e = 0, 1, 2
    powers = []
    for a in range(3):
        d = c[:, a].astype(float).reshape(shp) - u[a][None]
        powers.append((np.ones_like(d), d, d * d))
    out = np.zeros((len(MOMENT_EXPONENTS),) + pdf.shape[1:], dtype=np.result_type(pdf, u))
    for k, e in enumerate(MOMENT_EXPONENTS):
        out[k] = (pdf * powers[0][e[0]] * powers[1][e[1]] * powers[2][e[2]]).sum(axis=0)
    return out


def _shift_terms():
    """(k, k', binomial product, exponent difference) for all e' <= e."""
    E = MOMENT_EXPONENTS
    out = []
    for k, e in enumerate(E):
        for k2, e2 in enumerate(E):
            if np.all(e2 <= e):
                b = 1
                for a in range(3):
                    b *= comb(int(e[a]), int(e2[a]))
                out.append((k, k2, float(b), tuple(int(v) for v in (e - e2))))
    return out


_SHIFT_TERMS = _shift_terms()


def raw_from_central(kappa: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Binomial shift back to raw moments:
    m_e = sum_{e' <= e} prod_a C(e_a, e'_a) u_a^(e_a - e'_a) kappa_e'."""
    upow = [(np.ones_like(u[a]), u[a], u[a] * u[a]) for a in range(3)]
    m = np.zeros(kappa.shape, dtype=np.result_type(kappa, u))
    for k, k2, b, d in _SHIFT_TERMS:
        m[k] += b * upow[0][d[0]] * upow[1][d[1]] * upow[2][d[2]] * kappa[k2]
    return m


def central_from_raw(m: np.ndarray, u: np.ndarray) -> np.ndarray:
    """N(u): raw -> central moments (binomial shift with -u)."""
    return raw_from_central(m, -u)


def eq_scalar(psi, u, S):
    """h^eq / f^eq of Sec. 2.2 (Eq. for h_i^eq; same form for f^eq, Sec. 2.3):
    psi w_i [1 + c.u/c_s^2 + (c.u)^2/(2 c_s^4) - u.u/(2 c_s^2)]."""
    uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    out = np.empty((S.Q,) + psi.shape, dtype=np.result_type(psi, u))
    for i in range(S.Q):
        cu = S.c[i, 0] * u[0] + S.c[i, 1] * u[1] + S.c[i, 2] * u[2]
        out[i] = S.w[i] * psi * (1.0 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2))
    return out


def eq_hydro(p, u, S):
    """Incompressible (velocity-based) g^eq of Sec. 2.2:
    w_i (p* + [c.u/c_s^2 + (c.u)^2/(2 c_s^4) - u.u/(2 c_s^2)])."""
    uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    out = np.empty((S.Q,) + p.shape, dtype=np.result_type(p, u))
    for i in range(S.Q):
        cu = S.c[i, 0] * u[0] + S.c[i, 1] * u[1] + S.c[i, 2] * u[2]
        out[i] = S.w[i] * (p + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2))
    return out


def guo_source(u, a, S):
    """Guo source S_i = w_i [(c_i - u)/c_s^2 + (c_i.u) c_i / c_s^4] . a."""
    out = np.empty((S.Q,) + u.shape[1:], dtype=np.result_type(u, a))
    for i in range(S.Q):
        cu = S.c[i, 0] * u[0] + S.c[i, 1] * u[1] + S.c[i, 2] * u[2]
        acc = 0.0
        for k in range(3):
            acc = acc + ((S.c[i, k] - u[k]) / CS2 + cu * S.c[i, k] / (CS2 * CS2)) * a[k]
        out[i] = S.w[i] * acc
    return out


def cm_collide(gs, geq, src, u, omega2, omega_high=1.0, omega_all=None):
    """Central-moment collision of Sec. 2.2 (relaxation of K(u) g):
    kappa' = kappa - W (kappa - kappa^eq) + (I - W/2) kappa^F,  g' = K(u)^-1 kappa'.
    W = diag: omega2 (per cell) for second-order moments, omega_high for the
    others (orders 0 and 1 are conserved up to the force term whatever their
    rate).  ``omega_all`` forces one rate for every moment (single-rate test)."""
    S27 = stencil(27)
    k = central_moments(gs, u, S27.c)
    keq = central_moments(geq, u, S27.c)
    kF = central_moments(src, u, S27.c)
    post = np.empty(k.shape, dtype=np.result_type(k, keq, kF, omega2))
    for m, e in enumerate(MOMENT_EXPONENTS):
        order = int(e.sum())
        if omega_all is not None:
            w = omega_all
        elif order == 2:
            w = omega2
        else:
            w = omega_high
        post[m] = k[m] - w * (k[m] - keq[m]) + (1.0 - 0.5 * w) * kF[m]
    raw = raw_from_central(post, u)
    return np.tensordot(_minv27(), raw, axes=(1, 0))


_MINV27 = []


def _minv27():
    """M^-1 of the D3Q27 raw-moment matrix (inverted once)."""
    if not _MINV27:
        _MINV27.append(np.linalg.inv(raw_moment_matrix(stencil(27).c)))
    return _MINV27[0]


class OracleLBM:
    """Literal FP64 implementation on a (nx, ny, nz) box.

    Cell (i, j, k) has its centre at (i + 1/2, j + 1/2, k + 1/2); z walls are
    the box faces z = 0 and z = nz.  Droplet, heat-source and background-
    gradient positions are given in these coordinates; heater patches by
    integer cell index.
    ``origin``/``global_shape`` place the box inside a larger periodic lattice
    (used to check sampled cells of a large run: the box is then treated as
    periodic and only cells at least 2 x steps away from its x/y edges are
    meaningful).  Walls, when enabled, are at the box's z faces.
    """

    def __init__(self, nx, ny, nz, params, q_phase=15, thermal="D3Q7",
                 sources: Sequence = (), patches=None, origin=(0, 0, 0),
                 global_shape=None):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.p = params
        self.Sh = stencil(q_phase)
        self.S27 = stencil(27)
        self.thermal = thermal
        self.lb_thermal = thermal.startswith("D3Q")
        self.Sf = stencil(int(thermal[3:])) if self.lb_thermal else None
        self.walls = bool(params.walls_z)
        self.NX, self.NY, self.NZ = global_shape if global_shape else (nx, ny, nz)
        ox, oy, oz = origin
        # integer cell indices and cell-centre coordinates (cell k at k + 1/2;
        # walls, when present, are the box faces z = 0 and z = NZ).  Along a
        # periodic axis a box cell past the lattice's end is the lattice cell
        # of index k mod N: it gets that cell's position (heat sources,
        # patches, background gradient, first moments).
        zk = np.arange(nz) + oz
        if not self.walls:
            zk = zk % self.NZ
        Zi, Yi, Xi = np.meshgrid(zk, (np.arange(ny) + oy) % self.NY,
                                 (np.arange(nx) + ox) % self.NX, indexing="ij")
        self.Xi, self.Yi, self.Zi = Xi, Yi, Zi
        self.X, self.Y, self.Z = Xi + 0.5, Yi + 0.5, Zi + 0.5
        self.q = self._heat_source(sources, patches)
        self.time = 0
        self.h = self.g = self.f = self.T = None

    # ------------------------------------------------------------ inputs
    def _heat_source(self, sources, patches):
        """Eq. HeatSource summed over the sources (+ heater patches)."""
        q = np.zeros((self.nz, self.ny, self.nx))
        for s in sources:
            r2 = (self.X - s.x) ** 2 + (self.Y - s.y) ** 2 + (self.Z - s.z) ** 2
            val = s.Q * np.exp(-2.0 * r2 / (s.w * s.w))
            if math.isfinite(s.d):
                val = np.where(r2 <= s.d * s.d, val, 0.0)
            q = q + val
        if patches is not None:
            for k, I in enumerate(patches.intensity):
                m = ((self.Zi == patches.z)
                     & (self.Xi >= patches.x0[k]) & (self.Xi < patches.x0[k] + patches.sx)
                     & (self.Yi >= patches.y0[k]) & (self.Yi < patches.y0[k] + patches.sy))
                q = q + np.where(m, I, 0.0)
        return q

    def add_heat_field(self, q):
        """A given per-cell heat-source density (dense [z][y][x]) added to the
        source q_T of the energy equation (Sec. 2.3), on top of the Gaussian
        sources and heater patches."""
        self.q = self.q + np.asarray(q, dtype=np.float64).reshape(self.nz, self.ny, self.nx)

    def init_droplets(self, droplets: Iterable):
        """Initial state: phi = max_k tanh profiles (Sec. 3.1 initial profile,
        phi0 + (phiH - phiL)/2 tanh(r/(xi/2))), u = sum_k phi_k v_k,
        h = h^eq(phi, u), g = g^eq(0, u), f = f^eq(T0, u); T0 is the conduction
        profile between the walls, else 0."""
        p = self.p
        phi = np.zeros((self.nz, self.ny, self.nx))
        u = np.zeros((3, self.nz, self.ny, self.nx))
        for d in droplets:
            dx = self.X - d.cx
            dx = dx - self.NX * np.round(dx / self.NX)
            dy = self.Y - d.cy
            dy = dy - self.NY * np.round(dy / self.NY)
            dz = self.Z - d.cz
            if not self.walls:
                dz = dz - self.NZ * np.round(dz / self.NZ)
            r = np.sqrt(dx * dx + dy * dy + dz * dz)
            pk = 0.5 * (1.0 + np.tanh(2.0 * (d.R - r) / p.xi))
            phi = np.maximum(phi, pk)
            u[0] += pk * d.ux
            u[1] += pk * d.uy
            u[2] += pk * d.uz
        if self.walls:
            Tb = self.T_wall_bottom()
            T0 = Tb + (p.T_top - Tb) * self.Z / self.NZ
        else:
            T0 = np.zeros_like(phi)
        self.h = eq_scalar(phi, u, self.Sh)
        self.g = eq_hydro(np.zeros_like(phi), u, self.S27)
        if self.lb_thermal:
            self.f = eq_scalar(T0, u, self.Sf)
        else:
            self.T = T0.copy()
        self.time = 0

    def T_wall_bottom(self):
        """Bottom wall temperature above each column, shape (ny, nx):
        T_bottom + T_bottom_amp cos(omega x) at the cell centre x, with
        omega = 2 pi k / NX (the planar heated channel's heated wall, Sec. 3.1);
        uniform T_bottom when no modulation is set."""
        p = self.p
        X = self.X[0]
        amp = getattr(p, "T_bottom_amp", 0.0)
        k = getattr(p, "T_bottom_waves", 0)
        if amp == 0.0 or k == 0:
            return np.full(X.shape, float(p.T_bottom))
        return p.T_bottom + amp * np.cos(2.0 * math.pi * k * X / self.NX)

    # ------------------------------------------------------------ a1 stream
    def _pull(self, pdf, S, rule=None, Tb=0.0, Tt=0.0):
        """Pull streaming p*_i(x) = p_i(x - c_i) (periodic by np.roll); at z
        walls the half-way bounce-back p*_i = p_opp(i) (rule None) or the
        anti-bounce-back p*_i = -p_opp(i) + 2 w_i T_w (rule 'abb').

        Moving walls (tangential velocity u_w, Sec. 3.3 sheared channel): the
        populations coming off a wall take the wall's momentum, by the
        equilibrium's linear term: g*_i = g_opp(i) + 2 w_i (c_i . u_w) / c_s^2
        (rule 'g', velocity-based equilibrium) and h*_i = h_opp(i) + 2 w_i
        phi_0 (c_i . u_w) / c_s^2 (rule 'h'), phi_0 the zeroth moment of the
        pulled h without the correction (the corrections of a tangential wall
        cancel in it); the thermal anti-bounce-back takes the even part of
        the equilibrium, 2 w_i T_w [1 + (c_i . u_w)^2 / (2 c_s^4) - u_w^2 / (2 c_s^2)]."""
        p = self.p
        ub = tuple(getattr(p, "wall_u_bottom", (0.0, 0.0)))
        ut = tuple(getattr(p, "wall_u_top", (0.0, 0.0)))
        moving = any(v != 0.0 for v in ub + ut)
        out = np.empty_like(pdf)
        fixes = []
        for i in range(S.Q):
            cx, cy, cz = (int(v) for v in S.c[i])
            out[i] = np.roll(pdf[i], shift=(cz, cy, cx), axis=(0, 1, 2))
            if self.walls and cz != 0:
                zl = 0 if cz == 1 else -1
                Tw = Tb if cz == 1 else Tt
                uw = ub if cz == 1 else ut
                cu = cx * uw[0] + cy * uw[1]
                back = pdf[S.opp[i]][zl]
                if rule == "abb":
                    e = 1.0 + cu * cu / (2 * CS2 * CS2) - (uw[0] ** 2 + uw[1] ** 2) / (2 * CS2)
                    out[i][zl] = -back + 2.0 * S.w[i] * Tw * e
                else:
                    out[i][zl] = back
                    if moving and rule in ("g", "h") and cu != 0.0:
                        fixes.append((i, zl, 2.0 * S.w[i] * cu / CS2))
        if fixes:
            phi0 = out.sum(axis=0) if rule == "h" else None
            for i, zl, c in fixes:
                out[i][zl] = out[i][zl] + (c * phi0[zl] if rule == "h" else c)
        return out

    # ------------------------------------------------------------ a3 stencils
    def _pad(self, psi, kind):
        """One ghost layer: periodic wrap in x, y (and z without walls); at
        walls a mirror (phi) or the Dirichlet ghost 2 T_w - T (T)."""
        q = np.pad(psi, 1, mode="wrap")
        if self.walls:
            if kind == "mirror":
                # contact angle theta (through phi = 1): the ghost value g
                # beyond the wall makes the one-sided normal derivative of
                # the equilibrium profile, (a - g) = -k w (1 - w), k =
                # (4 / xi) cos theta, w = (a + g) / 2 the wall value, a the
                # first fluid cell (the wetting condition of the conservative
                # phase field); theta = 90 degrees gives the mirror g = a
                q[0] = self._wet_ghost(q[1], getattr(self.p, "theta_bottom", 90.0))
                q[-1] = self._wet_ghost(q[-2], getattr(self.p, "theta_top", 90.0))
            else:
                q[0] = 2.0 * np.pad(self.T_wall_bottom(), 1, mode="wrap") - q[1]
                q[-1] = 2.0 * self.p.T_top - q[-2]
        return q

    def _wet_ghost(self, a, theta_deg):
        """Ghost phi beyond a wall with contact angle theta: the root of
        g - a = k ((a + g)/2) (1 - (a + g)/2), k = (4 / xi) cos theta, that
        tends to g = a as k -> 0, in the form s = a + g = 4 a / ((1 - k/2) +
        sqrt((1 - k/2)^2 + 2 k a)) (no cancellation)."""
        if theta_deg == 90.0:
            return a.copy()
        k = 4.0 / self.p.xi * math.cos(math.radians(theta_deg))
        b = 1.0 - 0.5 * k
        s = 4.0 * a / (b + np.sqrt(np.maximum(b * b + 2.0 * k * a, 0.0)))
        return s - a

    def _at(self, q, c):
        """Value of a padded field at x + c for every interior x."""
        cx, cy, cz = (int(v) for v in c)
        return q[1 + cz:1 + cz + self.nz, 1 + cy:1 + cy + self.ny, 1 + cx:1 + cx + self.nx]

    def grad_iso(self, q):
        """Isotropic gradient (1/c_s^2) sum_i w_i c_i psi(x + c_i), D3Q27."""
        S = self.S27
        gx = np.zeros((self.nz, self.ny, self.nx))
        gy = np.zeros_like(gx)
        gz = np.zeros_like(gx)
        for i in range(S.Q):
            v = self._at(q, S.c[i])
            gx = gx + S.w[i] * S.c[i, 0] * v
            gy = gy + S.w[i] * S.c[i, 1] * v
            gz = gz + S.w[i] * S.c[i, 2] * v
        return np.stack([gx, gy, gz]) / CS2

    def lap_iso(self, q):
        """Isotropic Laplacian (2/c_s^2) sum_i w_i [psi(x + c_i) - psi(x)], D3Q27."""
        S = self.S27
        centre = self._at(q, (0, 0, 0))
        acc = np.zeros_like(centre)
        for i in range(S.Q):
            acc = acc + S.w[i] * (self._at(q, S.c[i]) - centre)
        return 2.0 * acc / CS2

    def grad_std(self, q):
        """Second-order central difference (psi(x+e) - psi(x-e)) / 2."""
        out = []
        for a in range(3):
            e = [0, 0, 0]
            e[a] = 1
            m = [0, 0, 0]
            m[a] = -1
            out.append(0.5 * (self._at(q, e) - self._at(q, m)))
        return np.stack(out)

    def lap_std(self, q):
        """7-point Laplacian sum_faces psi(x + e) - 6 psi(x)."""
        centre = self._at(q, (0, 0, 0))
        acc = np.zeros_like(centre)
        for e in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            acc = acc + self._at(q, e)
        return acc - 6.0 * centre

    # ------------------------------------------------------------ a2-a6
    def _background(self):
        G = self.p.grad_T
        o = self.p.grad_T_origin
        return G[0] * (self.X - o[0]) + G[1] * (self.Y - o[1]) + G[2] * (self.Z - o[2])

    def _macro_from_pulled(self, hs, gs, fs):
        p = self.p
        phi = hs.sum(axis=0)                       # Eq. zeroth_moment_phase
        pstar = gs.sum(axis=0)                     # Eq. zeroth_moment_hydro
        T = fs.sum(axis=0) if self.lb_thermal else self.T   # Eq. zeroth_moment_thermal
        qphi = self._pad(phi, "mirror")
        qT = self._pad(T, "dirichlet")
        gphi = self.grad_iso(qphi)
        lphi = self.lap_iso(qphi)
        G = np.array(p.grad_T).reshape(3, 1, 1, 1)
        gT = self.grad_iso(qT) + G
        Ttot = T + self._background()
        sigma = p.sigma_ref + p.sigma_T * (Ttot - p.T_ref)          # Eq. sigma(T)
        beta = 12.0 * sigma / p.xi
        kap = 1.5 * sigma * p.xi
        mu = 4.0 * beta * phi * (phi - 1.0) * (phi - 0.5) - kap * lphi
        g2 = gphi[0] ** 2 + gphi[1] ** 2 + gphi[2] ** 2
        gTgphi = gT[0] * gphi[0] + gT[1] * gphi[1] + gT[2] * gphi[2]
        Fs = mu * gphi + 1.5 * p.xi * p.sigma_T * (g2 * gT - gTgphi * gphi)  # Eq. F_s
        rho = p.rho_L + phi * (p.rho_H - p.rho_L)                   # Eq. rho(phi)
        Fb = rho * np.array(p.gravity).reshape(3, 1, 1, 1)           # Eq. F_b
        F = Fs + Fb
        jg = np.einsum("iq,i...->q...", self.S27.c.astype(float), gs)
        drho = p.rho_H - p.rho_L
        if drho != 0.0:
            F = F + self._density_ratio_forces(gs, pstar, phi, rho, gphi, jg, F)
        a = F / rho
        u = jg + 0.5 * a
        return dict(phi=phi, p=pstar, T=T, u=u, a=a, F=F, rho=rho, gphi=gphi,
                    lphi=lphi, gT=gT, g2=g2)

    def _density_ratio_forces(self, gs, pstar, phi, rho, gphi, jg, Fsb):
        """F_p + F_mu of Sec. 2.2 (the pressure and viscous correction forces
        of the velocity-based formulation, zero at density ratio 1):
          F_p  = -p* c_s^2 (rho_H - rho_L) grad phi,
          F_mu = nu (rho_H - rho_L) [grad u + (grad u)^T] . grad phi,
        nu = c_s^2 (tau(phi) - 1/2), tau(phi) = tau_L + phi (tau_H - tau_L).
        The strain rate comes from the non-equilibrium second moments of the
        pulled g (the paper's remark after the F_mu equation), by the
        Chapman-Enskog relation of the forced BGK/CM scheme,
          sum_i c_ia c_ib (g*_i - g^eq_i + S_i / 2) = -tau c_s^2 (d_a u_b + d_b u_a),
        with g^eq, the Guo source S and the velocity evaluated from the forces
        known before F_mu: u0 = j + a0 / 2, a0 = (F_s + F_b + F_p) / rho."""
        p = self.p
        drho = p.rho_H - p.rho_L
        Fp = -pstar * CS2 * drho * gphi
        a0 = (Fsb + Fp) / rho
        u0 = jg + 0.5 * a0
        neq = gs - eq_hydro(pstar, u0, self.S27) + 0.5 * guo_source(u0, a0, self.S27)
        c = self.S27.c.astype(float)
        Pi = np.einsum("ia,ib,i...->ab...", c, c, neq)
        tau = (p.nu_L / CS2 + 0.5) + phi * ((p.nu_H - p.nu_L) / CS2)
        strain = -Pi / (tau * CS2)
        nu = CS2 * (tau - 0.5)
        Fmu = nu * drho * np.einsum("ab...,b...->a...", strain, gphi)
        return Fp + Fmu

    # ------------------------------------------------------------ RK (a9')
    def kappa(self, phi):
        """Thermal conductivity, linear in phi (Sec. 2.3; the printed
        kappa_H + phi (kappa_H - kappa_L) read as kappa_L at phi = 0 and
        kappa_H at phi = 1)."""
        p = self.p
        return p.alpha_L + phi * (p.alpha_H - p.alpha_L)

    def heat_capacity(self, phi):
        """Volumetric heat capacity rho c_p of Eq. temperature, with rho and
        c_p each linear in phi (Eq. rho(phi); Sec. 2.3 for c_p, read like
        kappa)."""
        p = self.p
        return (p.rho_L + phi * (p.rho_H - p.rho_L)) * (p.cp_L + phi * (p.cp_H - p.cp_L))

    def heat_capacity_slope(self, phi):
        """d(rho c_p)/d phi."""
        p = self.p
        rho = p.rho_L + phi * (p.rho_H - p.rho_L)
        cp = p.cp_L + phi * (p.cp_H - p.cp_L)
        return (p.rho_H - p.rho_L) * cp + rho * (p.cp_H - p.cp_L)

    def varying_heat_capacity(self):
        p = self.p
        return p.cp_H != p.cp_L or p.rho_H != p.rho_L

    def alpha(self, phi):
        """Thermal diffusivity kappa / (rho c_p) of a cell."""
        return self.kappa(phi) / self.heat_capacity(phi)

    def rk_rhs(self, psi, u, phi):
        """R(T) = -u.(grad T + G) + alpha(phi) lap T
                  + (kappa_H - kappa_L) / (rho c_p) grad phi . (grad T + G) + q_T
        (Eq. temperature: (grad kappa . grad T_total + kappa lap T) / (rho c_p),
        where T_total = T + G.(x - x0) and lap of the linear background is
        zero); standard 7-point / central operators, or the isotropic D3Q27
        ones, for T and phi alike (phi mirrored at walls)."""
        p = self.p
        q = self._pad(psi, "dirichlet")
        qp = self._pad(phi, "mirror")
        if p.rk_isotropic_fd:
            gr, lp, gp = self.grad_iso(q), self.lap_iso(q), self.grad_iso(qp)
        else:
            gr, lp, gp = self.grad_std(q), self.lap_std(q), self.grad_std(qp)
        G = p.grad_T
        gt = [gr[k] + G[k] for k in range(3)]
        adv = u[0] * gt[0] + u[1] * gt[1] + u[2] * gt[2]
        C = self.heat_capacity(phi)
        cond = self.kappa(phi) / C * lp
        if p.alpha_H != p.alpha_L:
            cond = cond + (p.alpha_H - p.alpha_L) / C * (gp[0] * gt[0] + gp[1] * gt[1] + gp[2] * gt[2])
        return -adv + cond + self.q

    # ------------------------------------------------------------ step
    def macro(self):
        """Macroscopic fields of the current time level (what the next step
        computes from its pulled PDFs), without advancing."""
        hs = self._pull(self.h, self.Sh, "h")
        gs = self._pull(self.g, self.S27, "g")
        fs = (self._pull(self.f, self.Sf, "abb", self.T_wall_bottom(), self.p.T_top)
              if self.lb_thermal else None)
        return self._macro_from_pulled(hs, gs, fs)

    def step(self, n: int = 1):
        for _ in range(n):
            self._step1()

    def _step1(self):
        p = self.p
        hs = self._pull(self.h, self.Sh, "h")
        gs = self._pull(self.g, self.S27, "g")
        fs = (self._pull(self.f, self.Sf, "abb", self.T_wall_bottom(), p.T_top)
              if self.lb_thermal else None)
        m = self._macro_from_pulled(hs, gs, fs)
        phi, u, a = m["phi"], m["u"], m["a"]

        # a7: phase field, Eq. lb_interface with Eq. phasefieldforce as Guo source
        w_phi = 1.0 / (0.5 + p.mobility / CS2)
        gphi = m["gphi"]
        nrm = np.sqrt(m["g2"]) + p.eps_n
        Fphi = 4.0 * phi * (1.0 - phi) / p.xi * gphi / nrm
        heq = eq_scalar(phi, u, self.Sh)
        h_new = np.empty(hs.shape, dtype=np.result_type(hs, Fphi, heq))
        for i in range(self.Sh.Q):
            cF = self.Sh.c[i, 0] * Fphi[0] + self.Sh.c[i, 1] * Fphi[1] + self.Sh.c[i, 2] * Fphi[2]
            h_new[i] = hs[i] - w_phi * (hs[i] - heq[i]) + (1.0 - 0.5 * w_phi) * self.Sh.w[i] * cF

        # a8: hydrodynamics, central-moment collision with tau(phi)
        tau_L = p.nu_L / CS2 + 0.5
        tau_H = p.nu_H / CS2 + 0.5
        tau = tau_L + phi * (tau_H - tau_L)
        geq = eq_hydro(m["p"], u, self.S27)
        src = guo_source(u, a, self.S27)
        g_new = cm_collide(gs, geq, src, u, 1.0 / tau, p.omega_high)

        # a9 / a9': temperature
        G = p.grad_T
        uG = u[0] * G[0] + u[1] * G[1] + u[2] * G[2]
        if self.lb_thermal:
            # per-cell rate from alpha(phi) = kappa / (rho c_p); the LB
            # recovers div(alpha grad T) = alpha lap T + grad alpha . grad T.
            # Eq. temperature wants alpha lap T + grad kappa . (grad T + G) / C
            # (C = rho c_p), and grad kappa / C - grad alpha = alpha grad C / C,
            # so the source adds grad kappa . G / C and alpha (C' / C)
            # grad phi . grad T (grad T without the background)
            alpha = self.alpha(phi)
            w_T = 1.0 / (0.5 + alpha / CS2)
            src = self.q - uG
            gphi = m["gphi"]
            if p.alpha_H != p.alpha_L:
                src = src + (p.alpha_H - p.alpha_L) / self.heat_capacity(phi) * (
                    gphi[0] * G[0] + gphi[1] * G[1] + gphi[2] * G[2])
            if self.varying_heat_capacity():
                gT = [m["gT"][k] - G[k] for k in range(3)]
                src = src + alpha * self.heat_capacity_slope(phi) / self.heat_capacity(phi) * (
                    gphi[0] * gT[0] + gphi[1] * gT[1] + gphi[2] * gT[2])
            feq = eq_scalar(m["T"], u, self.Sf)
            f_new = np.empty(fs.shape, dtype=np.result_type(fs, feq, src, w_T))
            for i in range(self.Sf.Q):
                f_new[i] = fs[i] - w_T * (fs[i] - feq[i]) + self.Sf.w[i] * src
            self.f = f_new
        else:
            T = self.T
            if self.thermal == "RK2":
                K1 = self.rk_rhs(T, u, phi)
                self.T = T + self.rk_rhs(T + 0.5 * K1, u, phi)
            else:
                K1 = self.rk_rhs(T, u, phi)
                K2 = self.rk_rhs(T + 0.5 * K1, u, phi)
                K3 = self.rk_rhs(T + 0.5 * K2, u, phi)
                K4 = self.rk_rhs(T + K3, u, phi)
                self.T = T + K1 / 6.0 + K2 / 3.0 + K3 / 3.0 + K4 / 6.0
        self.h, self.g = h_new, g_new
        self.time += 1
        return m

    # ------------------------------------------------------------ a10
    def diagnostics(self) -> Dict[str, float]:
        """phi mass, sum T, kinetic energy 1/2 sum rho |u|^2, phi-weighted
        first moments and the centroid sum(phi x)/sum(phi) of the current level."""
        m = self.macro()
        phi, u, rho, T = m["phi"], m["u"], m["rho"], m["T"]
        mass = float(phi.sum())
        out = dict(mass=mass, heat=float(T.sum()),
                   kinetic=float(0.5 * (rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)).sum()),
                   mx=float((phi * self.X).sum()), my=float((phi * self.Y).sum()),
                   mz=float((phi * self.Z).sum()))
        out["centroid"] = (out["mx"] / mass, out["my"] / mass, out["mz"] / mass) if mass else (0, 0, 0)
        return out

    def state(self):
        s = dict(h=self.h.copy(), g=self.g.copy())
        if self.lb_thermal:
            s["f"] = self.f.copy()
        else:
            s["T"] = self.T.copy()
        return s


def build(workload, origin=(0, 0, 0), shape=None) -> OracleLBM:
    """Oracle instance for a ``workloads.Workload`` (optionally a sub-box)."""
    nx, ny, nz = shape if shape else (workload.nx, workload.ny, workload.nz)
    o = OracleLBM(nx, ny, nz, workload.params, workload.q_phase, workload.thermal,
                  workload.sources, workload.patches, origin=origin,
                  global_shape=(workload.nx, workload.ny, workload.nz))
    o.init_droplets(workload.droplets)
    return o
