"""Pins of the oracle's algebra against what the paper and mathematics fix:
stencil weights (App. B), isotropy, equilibrium moments (Sec. 2.2/2.3),
the central-moment transform (Sec. 2.2), the Guo source, and the
finite-difference operators (Sec. 2.4) on polynomials and sinusoids."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import model as om
from oracle.stencils import stencil

HERE = os.path.dirname(__file__)
RNG = np.random.Generator(np.random.PCG64(1234))


def _golden_weights():
    rows = {}
    with open(os.path.join(HERE, "golden", "stencil_weights.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, cls, cnt, wt = line.split()
            rows.setdefault(int(name[3:]), []).append((cls, int(cnt), Fraction(wt)))
    return rows


def _cls(c):
    n = int(np.abs(c).sum())
    return ["rest", "face", "edge", "corner"][n]


@pytest.mark.parametrize("Q", [7, 15, 19, 27])
def test_weights_match_appendix_b(Q):
    S = stencil(Q)
    gold = _golden_weights()[Q]
    assert S.Q == sum(cnt for _, cnt, _ in gold)
    for cls, cnt, wt in gold:
        idx = [i for i in range(Q) if _cls(S.c[i]) == cls]
        assert len(idx) == cnt
        assert all(S.w_exact[i] == wt for i in idx)
    # distinct velocities, opposite table
    assert len({tuple(v) for v in S.c}) == Q
    for i in range(Q):
        assert np.array_equal(S.c[S.opp[i]], -S.c[i])


@pytest.mark.parametrize("Q", [7, 15, 19, 27])
def test_isotropy(Q):
    S = stencil(Q)
    w = S.w_exact
    c = S.c
    assert sum(w) == 1
    for a in range(3):
        assert sum(w[i] * c[i, a] for i in range(Q)) == 0
        for b in range(3):
            m2 = sum(w[i] * c[i, a] * c[i, b] for i in range(Q))
            assert m2 == (Fraction(1, 3) if a == b else 0)   # c_s^2 = 1/3
    # fourth order: sum w c_x^2 c_y^2 = c_s^4 = 1/9 holds for Q15/19/27 only
    m22 = sum(w[i] * c[i, 0] ** 2 * c[i, 1] ** 2 for i in range(Q))
    m4 = sum(w[i] * c[i, 0] ** 4 for i in range(Q))
    if Q == 7:
        assert m22 == 0
    else:
        assert m22 == Fraction(1, 9) and m4 == Fraction(1, 3)


def test_moment_matrix_inverse_and_shift():
    S = stencil(27)
    M = om.raw_moment_matrix(S.c)
    Minv = np.linalg.inv(M)
    assert np.abs(Minv @ M - np.eye(27)).max() < 1e-14
    # N(u) N(-u) = I on random moment vectors (per cell u)
    u = RNG.uniform(-0.2, 0.2, size=(3, 5))
    m = RNG.standard_normal((27, 5))
    back = om.raw_from_central(om.central_from_raw(m, u), u)
    assert np.abs(back - m).max() < 1e-14


def test_central_moments_two_routes():
    """Definition sum_i g_i prod (c-u)^e equals N(u) M g, and K(u)^-1 built
    as M^-1 N(-u) equals a direct numerical inverse of K(u)."""
    S = stencil(27)
    M = om.raw_moment_matrix(S.c)
    u = RNG.uniform(-0.15, 0.15, size=3)
    g = RNG.standard_normal(27)
    k_def = om.central_moments(g.reshape(27, 1), u.reshape(3, 1), S.c)[:, 0]
    k_shift = om.central_from_raw((M @ g).reshape(27, 1), u.reshape(3, 1))[:, 0]
    assert np.abs(k_def - k_shift).max() < 1e-13
    # K(u) column by column from the definition
    K = np.stack([om.central_moments(np.eye(27)[:, j:j + 1], u.reshape(3, 1), S.c)[:, 0]
                  for j in range(27)], axis=1)
    Kinv_direct = np.linalg.inv(K)
    Kinv_route = np.stack([
        np.linalg.inv(M) @ om.raw_from_central(np.eye(27)[:, j:j + 1], u.reshape(3, 1))[:, 0]
        for j in range(27)], axis=1)
    assert np.abs(Kinv_direct - Kinv_route).max() < 1e-10


@pytest.mark.parametrize("Q", [7, 15, 19, 27])
def test_scalar_equilibrium_moments(Q):
    S = stencil(Q)
    psi = RNG.uniform(0, 1, size=7)
    u = RNG.uniform(-0.1, 0.1, size=(3, 7))
    eq = om.eq_scalar(psi, u, S)
    assert np.abs(eq.sum(0) - psi).max() < 1e-15
    for a in range(3):
        assert np.abs((S.c[:, a, None] * eq).sum(0) - psi * u[a]).max() < 1e-15


def test_hydro_equilibrium_moments():
    S = stencil(27)
    p = RNG.uniform(-1e-2, 1e-2, size=6)
    u = RNG.uniform(-0.1, 0.1, size=(3, 6))
    eq = om.eq_hydro(p, u, S)
    assert np.abs(eq.sum(0) - p).max() < 1e-16
    for a in range(3):
        assert np.abs((S.c[:, a, None] * eq).sum(0) - u[a]).max() < 1e-16
        for b in range(3):
            m2 = (S.c[:, a, None] * S.c[:, b, None] * eq).sum(0)
            want = p / 3.0 * (a == b) + u[a] * u[b]
            assert np.abs(m2 - want).max() < 1e-16


def test_guo_source_moments():
    S = stencil(27)
    u = RNG.uniform(-0.1, 0.1, size=(3, 4))
    a = RNG.uniform(-1e-3, 1e-3, size=(3, 4))
    s = om.guo_source(u, a, S)
    assert np.abs(s.sum(0)).max() < 1e-18
    for x in range(3):
        assert np.abs((S.c[:, x, None] * s).sum(0) - a[x]).max() < 1e-18
        for y in range(3):
            m2 = (S.c[:, x, None] * S.c[:, y, None] * s).sum(0)
            assert np.abs(m2 - (u[x] * a[y] + a[x] * u[y])).max() < 1e-18


def test_single_rate_cm_equals_bgk_guo():
    """With every moment relaxed at one rate the central-moment collision is
    the BGK update g - w (g - g^eq) + (1 - w/2) S exactly (K(u) is linear)."""
    S = stencil(27)
    n = 9
    u = RNG.uniform(-0.1, 0.1, size=(3, n))
    p = RNG.uniform(-1e-3, 1e-3, size=n)
    geq = om.eq_hydro(p, u, S)
    gs = geq + RNG.standard_normal((27, n)) * 1e-3
    src = om.guo_source(u, RNG.uniform(-1e-4, 1e-4, size=(3, n)), S)
    w = 1.37
    cm = om.cm_collide(gs, geq, src, u, omega2=None, omega_all=w)
    bgk = gs - w * (gs - geq) + (1 - 0.5 * w) * src
    assert np.abs(cm - bgk).max() < 1e-14


def test_cm_collision_conserves_and_forces():
    S = stencil(27)
    n = 11
    u = RNG.uniform(-0.1, 0.1, size=(3, n))
    a = RNG.uniform(-1e-4, 1e-4, size=(3, n))
    p = RNG.uniform(-1e-3, 1e-3, size=n)
    geq = om.eq_hydro(p, u, S)
    gs = geq + RNG.standard_normal((27, n)) * 1e-3
    # make u consistent with the Guo definition u = sum c g + a/2
    j = (S.c.T.astype(float) @ gs)
    gs_u = j + 0.5 * a
    geq = om.eq_hydro(gs.sum(0), gs_u, S)
    src = om.guo_source(gs_u, a, S)
    post = om.cm_collide(gs, geq, src, gs_u, omega2=RNG.uniform(0.6, 1.9, size=n))
    assert np.abs(post.sum(0) - gs.sum(0)).max() < 1e-15
    assert np.abs(S.c.T.astype(float) @ post - (j + a)).max() < 1e-15
    # second-order central moments relax at omega2, third+ are set to eq + F/2
    kp = om.central_moments(post, gs_u, S.c)
    keq = om.central_moments(geq, gs_u, S.c)
    kF = om.central_moments(src, gs_u, S.c)
    for m, e in enumerate(om.MOMENT_EXPONENTS):
        if e.sum() >= 3:
            assert np.abs(kp[m] - (keq[m] + 0.5 * kF[m])).max() < 1e-14


# ------------------------------------------------------------ FD operators
def _box(n=6):
    o = om.OracleLBM(n, n, n, __import__("workloads").Params(), 15, "D3Q7")
    return o


def _padded_poly(o, fn):
    z, y, x = np.meshgrid(np.arange(-1, o.nz + 1), np.arange(-1, o.ny + 1),
                          np.arange(-1, o.nx + 1), indexing="ij")
    return fn(x.astype(float), y.astype(float), z.astype(float))


def test_fd_exact_on_quadratics():
    o = _box()
    cf = RNG.standard_normal(10)

    def f(x, y, z):
        return (cf[0] + cf[1] * x + cf[2] * y + cf[3] * z + cf[4] * x * x + cf[5] * y * y
                + cf[6] * z * z + cf[7] * x * y + cf[8] * y * z + cf[9] * x * z)
    q = _padded_poly(o, f)
    x, y, z = o.Xi, o.Yi, o.Zi   # the padded polynomial uses cell indices
    gx = cf[1] + 2 * cf[4] * x + cf[7] * y + cf[9] * z
    gy = cf[2] + 2 * cf[5] * y + cf[7] * x + cf[8] * z
    gz = cf[3] + 2 * cf[6] * z + cf[8] * y + cf[9] * x
    lap = 2 * (cf[4] + cf[5] + cf[6])
    for grad, lapf in ((o.grad_iso, o.lap_iso), (o.grad_std, o.lap_std)):
        g = grad(q)
        assert np.abs(g[0] - gx).max() < 1e-12
        assert np.abs(g[1] - gy).max() < 1e-12
        assert np.abs(g[2] - gz).max() < 1e-12
        assert np.abs(lapf(q) - lap).max() < 1e-12


def test_fd_sinusoid_symbols():
    """On psi = sin(k.x) the D3Q27 isotropic Laplacian has the symbol
    -(2/c_s^2) sum_i w_i (1 - cos(k.c_i)); the 7-point one sum_a (2 cos k_a - 2)."""
    o = _box(8)
    k = np.array([2 * np.pi / 8, 2 * np.pi / 4, 0.3])
    q = _padded_poly(o, lambda x, y, z: np.sin(k[0] * x + k[1] * y + k[2] * z))
    psi = np.sin(k[0] * o.Xi + k[1] * o.Yi + k[2] * o.Zi)
    S = stencil(27)
    sym_iso = -(2 / om.CS2) * sum(S.w[i] * (1 - np.cos(k @ S.c[i])) for i in range(27))
    sym_std = sum(2 * np.cos(ka) - 2 for ka in k)
    assert np.abs(o.lap_iso(q) - sym_iso * psi).max() < 1e-13
    assert np.abs(o.lap_std(q) - sym_std * psi).max() < 1e-13
