"""The planar heated channel of Sec. 3.1 (App. A): two fluid layers between
walls, a flat interface, the lower wall at T_h + T_0 cos(omega x), the upper
at T_c.  At small Re, Ma and Ca the steady state is conduction in each layer
and Stokes flow driven by the Marangoni stress at the interface.

Two forms of the steady state are here, both written from the mathematics:

* ``solve``: conduction and Stokes flow solved layer by layer.  T: Laplace's
  equation in each layer with T and the heat flux k dT/dy continuous at the
  interface.  Flow: stream function psi = F(y) sin(omega x) with
  F = (A + B y) cosh(omega y) + (C + D y) sinh(omega y) in each layer; no
  slip at the walls, v = 0 and u continuous at the interface, and the
  tangential stress balance mu_a u_a' - mu_b u_b' = -d sigma / dx there.
  The eight coefficients come from one 8 x 8 linear solve.
* ``printed``: App. A's closed form.  Read with two corrections to its
  temperature: the y <= 0 and y > 0 branches of the cos(omega x) term are
  taken the other way round (as printed, neither branch meets its wall
  condition), and the lower layer's linear slope carries the factor k_r
  (flux continuity).  Its velocity is used as printed.

Coordinates: y is measured from the interface (upper layer a: 0 < y < a,
lower layer b: -b < y < 0); k_r = k_a / k_b, mu_r = mu_a / mu_b.
"""
import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Channel:
    a: float          # upper layer height
    b: float          # lower layer height
    omega: float      # wave number of the wall modulation
    T_h: float
    T_c: float
    T_0: float
    k_a: float
    k_b: float
    mu_a: float
    mu_b: float
    sigma_T: float

    @property
    def k_r(self):
        return self.k_a / self.k_b

    @property
    def mu_r(self):
        return self.mu_a / self.mu_b


def _basis(w, y):
    """F, F', F'' of the four stream-function basis functions at y."""
    c, s = math.cosh(w * y), math.sinh(w * y)
    F = [c, y * c, s, y * s]
    dF = [w * s, c + w * y * s, w * c, s + w * y * c]
    d2F = [w * w * c, 2 * w * s + w * w * y * c, w * w * s, 2 * w * c + w * w * y * s]
    return np.array(F), np.array(dF), np.array(d2F)


def _temperature_parts(ch):
    """Interface temperature, layer slopes and the cos(omega x) amplitude
    functions of the conduction solution."""
    w, a, b = ch.omega, ch.a, ch.b
    Ti = (ch.k_a * ch.T_c * b + ch.k_b * ch.T_h * a) / (ch.k_a * b + ch.k_b * a)
    s_a = (ch.T_c - Ti) / a
    s_b = (Ti - ch.T_h) / b
    # Y_a = A sinh(omega (a - y)); Y_b = C cosh(omega y) + D sinh(omega y)
    A = ch.T_0 / (math.sinh(w * a) * math.cosh(w * b) + ch.k_r * math.cosh(w * a) * math.sinh(w * b))
    C = A * math.sinh(w * a)
    D = -ch.k_r * A * math.cosh(w * a)
    return Ti, s_a, s_b, A, C, D


def solve(ch):
    """Returns functions T(x, y), u(x, y), v(x, y) of the layer-by-layer solution."""
    w, a, b = ch.omega, ch.a, ch.b
    Ti, s_a, s_b, A, C, D = _temperature_parts(ch)
    # Marangoni stress: d sigma/dx at y = 0 = sigma_T dT/dx = -sigma_T omega Y(0) sin(omega x)
    Y0 = A * math.sinh(w * a)
    M = np.zeros((8, 8))
    r = np.zeros(8)
    Fa_a, dFa_a, _ = _basis(w, a)
    Fb_b, dFb_b, _ = _basis(w, -b)
    F0, dF0, d2F0 = _basis(w, 0.0)
    M[0, :4] = Fa_a                   # v = 0 at the upper wall
    M[1, :4] = dFa_a                  # u = 0 at the upper wall
    M[2, 4:] = Fb_b                   # v = 0 at the lower wall
    M[3, 4:] = dFb_b                  # u = 0 at the lower wall
    M[4, :4] = F0                     # v = 0 on the interface (upper side)
    M[5, 4:] = F0                     # v = 0 on the interface (lower side)
    M[6, :4] = dF0                    # u continuous
    M[6, 4:] = -dF0
    M[7, :4] = ch.mu_a * d2F0         # mu_a u_a' - mu_b u_b' = -d sigma/dx
    M[7, 4:] = -ch.mu_b * d2F0
    r[7] = ch.sigma_T * w * Y0        # coefficient of sin(omega x)
    coef = np.linalg.solve(M, r)
    ca, cb = coef[:4], coef[4:]

    def T(x, y):
        x, y = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float))
        up = y > 0
        lin = np.where(up, Ti + s_a * y, Ti + s_b * y)
        Ya = A * np.sinh(w * (a - y))
        Yb = C * np.cosh(w * y) + D * np.sinh(w * y)
        return lin + np.where(up, Ya, Yb) * np.cos(w * x)

    def _F(y, k):
        y = np.asarray(y, float)
        cw, sw = np.cosh(w * y), np.sinh(w * y)
        if k == 0:
            parts = [cw, y * cw, sw, y * sw]
        else:
            parts = [w * sw, cw + w * y * sw, w * cw, sw + w * y * cw]
        fa = sum(ca[i] * parts[i] for i in range(4))
        fb = sum(cb[i] * parts[i] for i in range(4))
        return np.where(y > 0, fa, fb)

    def u(x, y):
        x, y = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float))
        return _F(y, 1) * np.sin(w * x)

    def v(x, y):
        x, y = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float))
        return -w * _F(y, 0) * np.cos(w * x)

    return T, u, v


def printed(ch):
    """App. A's closed form (temperature read as stated in the module
    docstring; velocity as printed, with mu_h = mu_a)."""
    w, a, b, kr = ch.omega, ch.a, ch.b, ch.k_r
    ar, br = a * w, b * w
    f = 1.0 / (kr * math.sinh(br) * math.cosh(ar) + math.sinh(ar) * math.cosh(br))
    Sa = math.sinh(ar) ** 2 - ar ** 2
    Sb = math.sinh(br) ** 2 - br ** 2
    C1a, C1b = math.sinh(ar) ** 2 / Sa, math.sinh(br) ** 2 / Sb
    C2a, C2b = -a * ar / Sa, -b * br / Sb
    C3a = (2 * ar - math.sinh(2 * ar)) / (2 * Sa)
    C3b = (-2 * br + math.sinh(2 * br)) / (2 * Sb)
    g = math.sinh(ar) * f
    h = (Sa * Sb) / (ch.mu_r * Sb * (math.sinh(2 * ar) - 2 * ar) + Sa * (math.sinh(2 * br) - 2 * br))
    Umax = -(ch.T_0 * ch.sigma_T / ch.mu_a) * g * h
    den = a + kr * b

    def T(x, y):
        x, y = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float))
        const = (kr * ch.T_c * b + ch.T_h * a) / den
        lin = np.where(y > 0, (ch.T_c - ch.T_h) * y / den, kr * (ch.T_c - ch.T_h) * y / den)
        up = ch.T_0 * f * np.sinh(ar - w * y)
        lo = ch.T_0 * f * (math.sinh(ar) * np.cosh(w * y) - kr * np.sinh(w * y) * math.cosh(ar))
        return const + lin + np.where(y > 0, up, lo) * np.cos(w * x)

    def u(x, y):
        x, y = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float))
        fa = (C1a + w * (C2a + C3a * y)) * np.cosh(w * y) + (C3a + w * C1a * y) * np.sinh(w * y)
        fb = (C1b + w * (C2b + C3b * y)) * np.cosh(w * y) + (C3b + w * C1b * y) * np.sinh(w * y)
        return Umax * np.where(y > 0, fa, fb) * np.sin(w * x)

    def v(x, y):
        x, y = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float))
        fa = C1a * y * np.cosh(w * y) + (C2a + C3a * y) * np.sinh(w * y)
        fb = C1b * y * np.cosh(w * y) + (C2b + C3b * y) * np.sinh(w * y)
        return -w * Umax * np.where(y > 0, fa, fb) * np.cos(w * x)

    return T, u, v


def l2(num, ref):
    """The relative l2 norm of Sec. 3.1: sqrt(sum (|num| - |ref|)^2 / sum |ref|^2)."""
    num, ref = np.abs(np.asarray(num)), np.abs(np.asarray(ref))
    return float(np.sqrt(((num - ref) ** 2).sum() / (ref ** 2).sum()))
