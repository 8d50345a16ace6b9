"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test pins one part of ``oracle/`` to something other than the oracle itself:
values printed in the paper (``tests/golden/paper_constants.json``), closed forms,
textbook radial reductions of the energies, symmetries that hold exactly on the
lattice, brute-force finite differences, and the Bogomolny bound. A plausible slip
in the oracle (a dropped term, a wrong sign, a swapped dx/dy, a wrong RK4 weight)
fails at least one of them. Unequal spacings are used where a test allows it.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2603_24370_gb300 import inputs as I

AH, CM, HARM = O.ABELIAN_HIGGS, O.CHIRAL_MAGNET, O.HARMONIC_TEST
BS = O.BABY_SKYRME
BS_PRM = (1.0, 0.7, 0.3)  # kappa, mu, nu
BEC = O.BEC
BEC_PRM = (1.3, 0.6, 2.0)  # g, Omega, mu
SID = O.SID
SID_PRM = (-1.0, -0.6, 0.5, 0.4, 0.3, 0.15, 0.35)  # a1, a2, b1, b2, b3, b4, nu
CMD = O.CM_DEMAG
CMD_PRM = (1.0, 0.8, 0.15, 0.5, 0.0, 0.7)  # J, D, K, h, dmi_type, mu_d
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")
AH_PRM = (1.0, 1.0)
CM_PRM = (1.0, 1.0, 0.1, 0.6, 0.0)


def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def grid(nx, ny, dx, dy):
    x = (np.arange(nx) - 0.5 * (nx - 1)) * dx
    y = (np.arange(ny) - 0.5 * (ny - 1)) * dy
    return np.meshgrid(x, y)


# ---------------------------------------------------------------- stencils (Eq. 1, Eq. 2)
def test_stencil_weights_are_the_papers():
    g = golden()
    nx, ny, dx, dy = 11, 11, 0.3, 0.7
    p = np.zeros((ny, nx))
    i0, j0 = 5, 5
    p[j0, i0] = 1.0
    d = O.derivatives(p, dx, dy)
    w1 = g["eq1_first_derivative"]
    w2 = g["eq2_second_derivative"]
    for off, w in zip(w1["offsets"], w1["weights"]):
        # d1x(i) = sum_m w_m p(i+m) / (12 dx)  ->  at i = i0 - m it equals w_m / (12 dx)
        assert d["fx"][j0, i0 - off] == pytest.approx(w / (w1["denominator"] * dx), abs=1e-15)
        assert d["fy"][j0 - off, i0] == pytest.approx(w / (w1["denominator"] * dy), abs=1e-15)
    for off, w in zip(w2["offsets"], w2["weights"]):
        assert d["fxx"][j0, i0 - off] == pytest.approx(w / (w2["denominator"] * dx * dx), abs=1e-13)
        assert d["fyy"][j0 - off, i0] == pytest.approx(w / (w2["denominator"] * dy * dy), abs=1e-13)
    # mixed derivative = product of the Eq. 1 weights in x and y
    for ox, wx in zip(w1["offsets"], w1["weights"]):
        for oy, wy in zip(w1["offsets"], w1["weights"]):
            exp = wx * wy / (144.0 * dx * dy)
            assert d["fxy"][j0 - oy, i0 - ox] == pytest.approx(exp, abs=1e-13)


def test_courant_number_is_the_papers():
    c = golden()["courant_number"]["value"]
    assert O.time_step(0.1, 0.1) == pytest.approx(c * 0.1, rel=1e-15)
    assert O.time_step(0.3, 0.2) == pytest.approx(c * 0.2, rel=1e-15)


def test_stencils_exact_on_polynomials():
    nx, ny, dx, dy = 13, 11, 0.37, 0.23
    X, Y = grid(nx, ny, dx, dy)
    f = 0.3 * X**4 - 1.1 * X**3 + 0.7 * X * X + 2.0 * X + 1.5 * Y**4 - 0.4 * Y**3 + 0.9 * X**3 * Y**2 + 0.2 * X * Y**4
    fx = 1.2 * X**3 - 3.3 * X * X + 1.4 * X + 2.0 + 2.7 * X * X * Y * Y + 0.2 * Y**4
    fy = 6.0 * Y**3 - 1.2 * Y * Y + 1.8 * X**3 * Y + 0.8 * X * Y**3
    fxx = 3.6 * X * X - 6.6 * X + 1.4 + 5.4 * X * Y * Y
    fyy = 18.0 * Y * Y - 2.4 * Y + 1.8 * X**3 + 2.4 * X * Y * Y
    fxy = 5.4 * X * X * Y + 0.8 * Y**3
    d = O.derivatives(f, dx, dy)
    sl = (slice(2, ny - 2), slice(2, nx - 2))
    for key, ref in (("fx", fx), ("fy", fy), ("fxx", fxx), ("fyy", fyy), ("fxy", fxy)):
        np.testing.assert_allclose(d[key][sl], ref[sl], rtol=0, atol=1e-9 * np.abs(ref).max(), err_msg=key)


def test_stencils_fourth_order():
    errs = []
    for n in (33, 65):
        L = 4.0
        dx = L / (n - 1)
        dy = 0.8 * dx
        X, Y = grid(n, n, dx, dy)
        f = np.sin(1.3 * X + 0.4) * np.cos(0.9 * Y - 0.2)
        ex = {
            "fx": 1.3 * np.cos(1.3 * X + 0.4) * np.cos(0.9 * Y - 0.2),
            "fy": -0.9 * np.sin(1.3 * X + 0.4) * np.sin(0.9 * Y - 0.2),
            "fxx": -1.69 * f,
            "fyy": -0.81 * f,
            "fxy": -1.17 * np.cos(1.3 * X + 0.4) * np.sin(0.9 * Y - 0.2),
        }
        d = O.derivatives(f, dx, dy)
        errs.append({k: np.abs(d[k] - ex[k])[2:-2, 2:-2].max() for k in ex})
    for k in errs[0]:
        ratio = errs[0][k] / errs[1][k]
        assert 12.0 < ratio < 20.0, (k, ratio)


# ---------------------------------------------------------------- energy (Table 1, Eq. 5)
def _ah_radial_energy(lam):
    from scipy.integrate import quad

    def integrand(r):
        t = math.tanh(r)
        s2 = 1.0 - t * t
        g, gp, a, ap = t, s2, t * t, 2.0 * t * s2
        return (0.5 * (gp * gp + g * g * (1 - a) ** 2 / (r * r)) + 0.5 * (ap / r) ** 2
                + lam / 8.0 * (1 - g * g) ** 2) * r

    val, _ = quad(integrand, 0.0, 40.0, epsabs=1e-13, epsrel=1e-13, limit=400)
    return 2 * math.pi * val


@pytest.mark.parametrize("lam", [1.0, 1.7])
def test_ah_energy_matches_radial_reduction(lam):
    """E_h of the radial vortex psi = tanh(r) e^{i theta}, A = tanh(r)^2 dtheta converges
    at fourth order to the textbook radial integral of Table 1's functional."""
    Econt = _ah_radial_energy(lam)
    errs = []
    for n in (81, 161):
        L = 20.0
        dx = L / (n - 1)
        f = O.ansatz(AH, [[0.0, 0.0, 1.0, 1.0, 0.0]], n, n, dx, dx)
        errs.append(abs(O.energy(AH, (lam, 1.0), f, dx, dx) - Econt))
    # a wrong term would make E_h converge to another value and the ratio collapse to ~1
    assert errs[1] < 1e-4 * Econt
    assert 12.0 < errs[0] / errs[1] < 20.0


def _cm_radial_energy(prm, w, helicity):
    from scipy.integrate import quad
    J, D, K, h = prm[:4]

    def integrand(r):
        f = math.pi * (1 - math.tanh(r / w))
        fp = -math.pi / w / math.cosh(r / w) ** 2
        ex = 0.5 * J * (fp * fp + math.sin(f) ** 2 / (r * r))
        dmi = D * math.cos(helicity) * (fp + math.sin(f) * math.cos(f) / r)
        return (ex + dmi + K * math.sin(f) ** 2 + h * (1 - math.cos(f))) * r

    val, _ = quad(integrand, 0.0, 60.0, epsabs=1e-13, epsrel=1e-13, limit=400)
    return 2 * math.pi * val


@pytest.mark.parametrize("helicity", [0.0, math.pi, 0.5 * math.pi])
def test_cm_energy_matches_radial_reduction(helicity):
    """Interfacial-DMI chiral magnet energy of a smooth skyrmion profile converges at
    fourth order to the radial reduction (Neel helicity: DMI = D cos(gamma)(f' + sin f cos f / r))."""
    w = 2.0
    Econt = _cm_radial_energy(CM_PRM, w, helicity)
    errs = []
    for n in (161, 321):
        L = 32.0
        dx = L / (n - 1)
        X, Y = grid(n, n, dx, dx)
        r = np.hypot(X, Y)
        th = np.arctan2(Y, X) + helicity
        f = np.pi * (1 - np.tanh(r / w))
        field = np.stack([np.sin(f) * np.cos(th), np.sin(f) * np.sin(th), np.cos(f)])
        errs.append(abs(O.energy(CM, CM_PRM, field, dx, dx) - Econt))
    assert errs[1] < 5e-5 * max(10.0, abs(Econt))
    assert 12.0 < errs[0] / errs[1] < 20.0


def test_dmi_sign_of_neel_skyrmion():
    """With D > 0 and interfacial DMI the Neel helicity 0 lowers the energy and helicity pi raises it."""
    n, dx = 64, 0.2
    for gam, sign in ((0.0, -1.0), (math.pi, 1.0)):
        f = O.ansatz(CM, [[0.0, 0.0, 1.0, 2.0, gam]], n, n, dx, dx)
        e_d = O.energy(CM, (1.0, 1.0, 0.1, 0.6, 0.0), f, dx, dx) - O.energy(CM, (1.0, 0.0, 0.1, 0.6, 0.0), f, dx, dx)
        assert sign * e_d > 0.5


def test_vacua_have_zero_energy_and_force():
    n, dx, dy = 16, 0.3, 0.2
    ah = np.zeros((4, n, n))
    ah[0] = math.cos(0.7)
    ah[1] = math.sin(0.7)
    assert abs(O.energy(AH, AH_PRM, ah, dx, dy)) < 1e-28  # |psi|^2 = 1 up to rounding
    assert np.abs(O.force(AH, AH_PRM, ah, dx, dy)).max() < 1e-13
    cm = np.zeros((3, n, n))
    cm[2] = 1.0
    assert O.energy(CM, CM_PRM, cm, dx, dy) == 0.0
    assert np.abs(O.force(CM, CM_PRM, cm, dx, dy)).max() == 0.0


def test_uniform_fields_closed_form():
    """Uniform fields: only the potential survives; E_h = area(I) * potential."""
    nx, ny, dx, dy = 14, 10, 0.3, 0.2
    area = (nx - 4) * (ny - 4) * dx * dy
    ah = np.zeros((4, ny, nx))
    ah[0] = 0.6
    ah[2] = 0.4  # a constant A is a pure gauge field: no energy of its own, but |D psi|^2 = A^2 |psi|^2
    lam, u = 1.3, 1.1
    exp = area * (0.5 * 0.4**2 * 0.36 + lam / 8 * (u * u - 0.36) ** 2)
    assert O.energy(AH, (lam, u), ah, dx, dy) == pytest.approx(exp, rel=1e-13)
    cm = np.zeros((3, ny, nx))
    cm[2] = -1.0
    K, h = 0.1, 0.6
    assert O.energy(CM, (1.0, 1.0, K, h, 0.0), cm, dx, dy) == pytest.approx(area * 2 * h, rel=1e-13)


def _rot90_scalar(a):
    # (x, y) -> (-y, x) about the array centre: new[j, i] = old[n-1-i, j]
    return a[::-1, :].T.copy()


def test_exact_90_degree_symmetry_ah():
    """Rotating space and A by 90 degrees maps the lattice onto itself: E_h is invariant
    and G is equivariant to rounding (Table 1's functional is rotation invariant)."""
    n, dx = 24, 0.25
    f = I.smooth_field(AH, n, n, dx, dx, seed=11)
    g = np.stack([_rot90_scalar(f[0]), _rot90_scalar(f[1]), -_rot90_scalar(f[3]), _rot90_scalar(f[2])])
    assert O.energy(AH, AH_PRM, g, dx, dx) == pytest.approx(O.energy(AH, AH_PRM, f, dx, dx), rel=1e-13)
    Gf, Gg = O.force(AH, AH_PRM, f, dx, dx), O.force(AH, AH_PRM, g, dx, dx)
    Grot = np.stack([_rot90_scalar(Gf[0]), _rot90_scalar(Gf[1]), -_rot90_scalar(Gf[3]), _rot90_scalar(Gf[2])])
    np.testing.assert_allclose(Gg, Grot, rtol=0, atol=1e-11 * np.abs(Gf).max())


def test_exact_90_degree_symmetry_cm_interfacial():
    """Interfacial DMI is invariant under a joint rotation of space and spin about e_3."""
    n, dx = 24, 0.25
    f = I.smooth_field(CM, n, n, dx, dx, seed=12)
    g = np.stack([-_rot90_scalar(f[1]), _rot90_scalar(f[0]), _rot90_scalar(f[2])])
    assert O.energy(CM, CM_PRM, g, dx, dx) == pytest.approx(O.energy(CM, CM_PRM, f, dx, dx), rel=1e-13)
    Gf, Gg = O.force(CM, CM_PRM, f, dx, dx), O.force(CM, CM_PRM, g, dx, dx)
    Grot = np.stack([-_rot90_scalar(Gf[1]), _rot90_scalar(Gf[0]), _rot90_scalar(Gf[2])])
    np.testing.assert_allclose(Gg, Grot, rtol=0, atol=1e-11 * np.abs(Gf).max())


def test_gauge_invariance_fourth_order():
    """psi -> psi e^{i chi}, A -> A + grad chi leaves Table 1's functional invariant; on
    the lattice E_h changes at O(h^4) and G_psi rotates with psi while G_A is unchanged."""
    errs_e, errs_g = [], []
    for n in (41, 81):
        L = 8.0
        dx = L / (n - 1)
        dy = 0.9 * dx
        X, Y = grid(n, n, dx, dy)
        f = I.smooth_field(AH, n, n, dx, dy, seed=5)
        chi = 0.8 * np.sin(0.6 * X + 0.3) * np.cos(0.5 * Y) + 0.1 * X * Y
        cx = 0.48 * np.cos(0.6 * X + 0.3) * np.cos(0.5 * Y) + 0.1 * Y
        cy = -0.4 * np.sin(0.6 * X + 0.3) * np.sin(0.5 * Y) + 0.1 * X
        c, s = np.cos(chi), np.sin(chi)
        g = np.stack([c * f[0] - s * f[1], s * f[0] + c * f[1], f[2] + cx, f[3] + cy])
        errs_e.append(abs(O.energy(AH, AH_PRM, g, dx, dy) - O.energy(AH, AH_PRM, f, dx, dy)))
        Gf, Gg = O.force(AH, AH_PRM, f, dx, dy), O.force(AH, AH_PRM, g, dx, dy)
        rot = np.stack([c * Gf[0] - s * Gf[1], s * Gf[0] + c * Gf[1], Gf[2], Gf[3]])
        errs_g.append(np.abs(Gg - rot)[:, 2:-2, 2:-2].max())
    assert errs_e[0] / errs_e[1] > 12.0 and errs_e[1] < 2e-4
    assert errs_g[0] / errs_g[1] > 12.0 and errs_g[1] < 1e-2


# ---------------------------------------------------------------- Baby Skyrme (Table 1)
def _bs_radial_energy(prm, w, N):
    """2 pi int r dr [1/2 (f'^2 + N^2 sin^2 f / r^2) + kappa^2/2 N^2 sin^2 f f'^2 / r^2
    + mu^2 (1 - cos f)] + pi int r dr nu^2/2 sin^2 f  (m_1^2 averages to sin^2 f / 2)."""
    from scipy.integrate import quad
    kappa, mu, nu = prm

    def integrand(r):
        f = math.pi * math.exp(-(r / w) ** 2)
        fp = -2.0 * r / (w * w) * f
        s2 = math.sin(f) ** 2
        sig = 0.5 * (fp * fp + N * N * s2 / (r * r))
        sky = 0.5 * kappa * kappa * N * N * s2 * fp * fp / (r * r)
        pot = mu * mu * (1.0 - math.cos(f)) + 0.25 * nu * nu * s2
        return (sig + sky + pot) * r

    val, _ = quad(integrand, 1e-12, 40.0, epsabs=1e-13, epsrel=1e-13, limit=400)
    return 2 * math.pi * val


@pytest.mark.parametrize("N,prm", [(1, (1.0, 0.7, 0.0)), (2, (0.8, 0.5, 0.6))])
def test_bs_energy_matches_radial_reduction(N, prm):
    """Lattice energy of a smooth hedgehog m = (sin f cos N theta, sin f sin N theta, cos f),
    f = pi exp(-r^2/w^2), converges at fourth order to the radial reduction of Table 1's
    Baby Skyrme functional (Skyrme term kappa^2/2 |d_1 m x d_2 m|^2)."""
    w = 2.5
    Econt = _bs_radial_energy(prm, w, N)
    errs = []
    for n in (121, 241):
        L = 24.0
        dx = L / (n - 1)
        X, Y = grid(n, n, dx, dx)
        r = np.hypot(X, Y)
        th = N * np.arctan2(Y, X)
        f = np.pi * np.exp(-(r / w) ** 2)
        field = np.stack([np.sin(f) * np.cos(th), np.sin(f) * np.sin(th), np.cos(f)])
        errs.append(abs(O.energy(BS, prm, field, dx, dx) - Econt))
    assert errs[1] < 2e-5 * Econt
    assert 12.0 < errs[0] / errs[1] < 20.0


def test_bs_skyrme_term_vanishes_on_one_dimensional_fields():
    """For m = m(x) the vectors d_1 m and d_2 m are parallel (d_2 m = 0): E_h and G do
    not depend on kappa at all."""
    nx, ny, dx, dy = 30, 20, 0.3, 0.25
    x = (np.arange(nx) - 0.5 * (nx - 1)) * dx
    T = 0.4 + 0.9 * np.sin(0.5 * x)
    P = 0.7 * np.cos(0.3 * x)
    f = np.stack([np.broadcast_to(v, (ny, nx)) for v in (np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T))])
    E = [O.energy(BS, (k, 0.6, 0.4), f, dx, dy) for k in (0.0, 1.3)]
    G = [O.force(BS, (k, 0.6, 0.4), f, dx, dy) for k in (0.0, 1.3)]
    assert E[1] == pytest.approx(E[0], rel=1e-14)
    np.testing.assert_allclose(G[1], G[0], rtol=0, atol=1e-13 * np.abs(G[0]).max())
    # and the kappa term is not zero in general
    g2 = I.smooth_field(BS, nx, ny, dx, dy, seed=9)
    assert O.energy(BS, (1.3, 0.6, 0.4), g2, dx, dy) > O.energy(BS, (0.0, 0.6, 0.4), g2, dx, dy) + 1e-3


def test_bs_uniform_fields_and_vacuum():
    nx, ny, dx, dy = 14, 10, 0.3, 0.2
    area = (nx - 4) * (ny - 4) * dx * dy
    kappa, mu, nu = 1.1, 0.7, 0.45
    m = np.array([0.48, -0.6, 0.64])
    f = np.broadcast_to(m[:, None, None], (3, ny, nx)).copy()
    exp = area * (mu * mu * (1 - m[2]) + 0.5 * nu * nu * m[0] ** 2)
    assert O.energy(BS, (kappa, mu, nu), f, dx, dy) == pytest.approx(exp, rel=1e-13)
    # force of a uniform field: the tangent part of dV/dm = (nu^2 m_1, 0, -mu^2)
    g = np.array([nu * nu * m[0], 0.0, -mu * mu])
    g = g - g.dot(m) * m
    G = O.force(BS, (kappa, mu, nu), f, dx, dy)
    np.testing.assert_allclose(G[:, 2:-2, 2:-2], np.broadcast_to(g[:, None, None], (3, ny - 4, nx - 4)), atol=1e-14)
    vac = np.zeros((3, ny, nx))
    vac[2] = 1.0
    assert O.energy(BS, (kappa, mu, nu), vac, dx, dy) == 0.0
    assert np.abs(O.force(BS, (kappa, mu, nu), vac, dx, dy)).max() == 0.0


def test_bs_exact_symmetries():
    """Table 1's Baby Skyrme functional is invariant under a joint rotation of space and
    spin about e_3 when nu = 0 (90 degrees), and under the 180-degree one for any nu."""
    n, dx = 24, 0.25
    f = I.smooth_field(BS, n, n, dx, dx, seed=13)
    g90 = np.stack([-_rot90_scalar(f[1]), _rot90_scalar(f[0]), _rot90_scalar(f[2])])
    prm0 = (1.2, 0.6, 0.0)
    assert O.energy(BS, prm0, g90, dx, dx) == pytest.approx(O.energy(BS, prm0, f, dx, dx), rel=1e-13)
    Gf, Gg = O.force(BS, prm0, f, dx, dx), O.force(BS, prm0, g90, dx, dx)
    Grot = np.stack([-_rot90_scalar(Gf[1]), _rot90_scalar(Gf[0]), _rot90_scalar(Gf[2])])
    np.testing.assert_allclose(Gg, Grot, rtol=0, atol=1e-11 * np.abs(Gf).max())
    r180 = lambda a: _rot90_scalar(_rot90_scalar(a))
    g180 = np.stack([-r180(f[0]), -r180(f[1]), r180(f[2])])
    assert O.energy(BS, BS_PRM, g180, dx, dx) == pytest.approx(O.energy(BS, BS_PRM, f, dx, dx), rel=1e-13)
    # with nu > 0 the 90-degree rotation is not a symmetry
    assert abs(O.energy(BS, BS_PRM, g90, dx, dx) - O.energy(BS, BS_PRM, f, dx, dx)) > 1e-6


def _bs_hedgehog_minimum(kappa, mu):
    """Energy of the charge-1 hedgehog minimum from the radial Euler-Lagrange ODE of
    2 pi int r dr [f'^2/2 + sin^2 f/(2 r^2) + kappa^2 sin^2 f f'^2/(2 r^2) + mu^2 (1 - cos f)],
    f(0) = pi, f -> 0: shooting on f'(0) by bisection, then quadrature."""
    from scipy.integrate import quad, solve_ivp
    k2, m2 = kappa * kappa, mu * mu

    def rhs(r, y):
        f, fp = y
        s, c = math.sin(f), math.cos(f)
        num = -fp + k2 * s * s * fp / (r * r) - k2 * s * c * fp * fp / r + s * c / r + m2 * r * s
        return [fp, num / (r + k2 * s * s / r)]

    def shoot(slope):
        r0 = 1e-4
        crosses = lambda r, y: y[0]
        return solve_ivp(rhs, (r0, 14.0), [math.pi - slope * r0, -slope], rtol=1e-11, atol=1e-13,
                         dense_output=True, events=[crosses])

    lo, hi = 0.1, 5.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if shoot(mid).t_events[0].size:
            hi = mid
        else:
            lo = mid
    sol = shoot(lo)
    rs = np.linspace(1e-4, sol.t[-1], 20000)
    rcut = rs[np.argmin(np.abs(sol.sol(rs)[0]))]

    def dens(r):
        f, fp = sol.sol(r)
        s2 = math.sin(f) ** 2
        return r * (0.5 * (fp * fp + s2 / (r * r)) + 0.5 * k2 * s2 * fp * fp / (r * r) + m2 * (1 - math.cos(f)))

    return 2 * math.pi * quad(dens, 1e-4, rcut, limit=500, epsabs=1e-12, epsrel=1e-12)[0]


@pytest.mark.slow
def test_bs_skyrmion_relaxes_to_the_radial_minimum():
    """The arrested flow relaxes a compact charge-1 ansatz to the baby skyrmion: its
    energy converges at fourth order in dx to the minimum of the radial reduction
    (independent shooting solution), above the bound 4 pi |Q| of the sigma-model term,
    with the charge exact and |m| = 1."""
    prm = (1.0, 0.7, 0.0)
    Eref = _bs_hedgehog_minimum(prm[0], prm[1])
    assert 4 * math.pi < Eref < 3 * 4 * math.pi
    errs = []
    for n, dx in ((96, 0.2), (192, 0.1)):
        f = O.ansatz(BS, [[0.0, 0.0, 1.0, 2.5, 0.0]], n, n, dx, dx)
        r = O.minimise(BS, prm, f, dx, dx, tol=1e-7, max_steps=20000)
        assert r["converged"]
        o = O.observables(BS, prm, r["f"], dx, dx)
        assert o["charge"] == pytest.approx(-1.0, abs=1e-10)
        assert o["norm_dev"] < 1e-14
        errs.append(abs(o["energy"] - Eref))
    assert errs[1] < 1e-4 * Eref
    assert 12.0 < errs[0] / errs[1] < 20.0


# ---------------------------------------------------------------- rotating BEC (Table 1)
def _bec_radial(w, m, r):
    """f(r) = (r / w)^|m| exp(-r^2 / w^2) and f'(r)."""
    f = (r / w) ** abs(m) * math.exp(-(r / w) ** 2)
    fp = f * (abs(m) / r - 2.0 * r / (w * w)) if r > 0 else 0.0
    return f, fp


@pytest.mark.parametrize("m", [0, 1, 2])
def test_bec_energy_and_rotation_match_the_radial_reduction(m):
    """psi = f(r) e^{i m theta}: the lattice energy converges at fourth order to
    2 pi int r dr [(f'^2 + m^2 f^2 / r^2)/2 + r^2 f^2 / 2 + g f^4 / 2 - mu f^2] - Omega m N,
    and the angular momentum Re int psi* L_z psi to m N (L_z = -i d_theta)."""
    from scipy.integrate import quad
    g, Om, mu = BEC_PRM
    w = 2.0

    def dens(r):
        f, fp = _bec_radial(w, m, r)
        kin = 0.5 * (fp * fp + (m * m * f * f / (r * r) if r > 0 else 0.0))
        return r * (kin + 0.5 * r * r * f * f + 0.5 * g * f ** 4 - mu * f * f)

    N = 2 * math.pi * quad(lambda r: r * _bec_radial(w, m, r)[0] ** 2, 0, 30, epsabs=1e-14, epsrel=1e-13)[0]
    Econt = 2 * math.pi * quad(dens, 0, 30, epsabs=1e-13, epsrel=1e-13, limit=400)[0] - Om * m * N
    errs, lz = [], []
    for n in (81, 161):
        L = 16.0
        dx = L / (n - 1)
        X, Y = grid(n, n, dx, dx)
        r = np.hypot(X, Y)
        f = (r / w) ** abs(m) * np.exp(-(r / w) ** 2)
        th = m * np.arctan2(Y, X)
        psi = np.stack([f * np.cos(th), f * np.sin(th)])
        errs.append(abs(O.energy(BEC, BEC_PRM, psi, dx, dx) - Econt))
        o = O.observables(BEC, BEC_PRM, psi, dx, dx)
        lz.append(abs(o["angular_momentum"] - m * o["atoms"]) + abs(o["atoms"] - N))
    assert errs[1] < 3e-5 * max(1.0, abs(Econt))
    assert 12.0 < errs[0] / errs[1] < 20.0
    assert lz[1] < 1e-4 * N
    if m:
        assert 12.0 < lz[0] / lz[1] < 20.0


def test_bec_symmetries():
    """The functional is invariant under a global phase (exactly: psi -> e^{i a} psi
    rotates G with psi) and, on a centred square grid, under 90-degree rotations of
    space (trap and L_z are rotation invariant)."""
    n, dx = 40, 0.3
    f = I.smooth_field(BEC, n, n, dx, dx, seed=17)
    a = 0.83
    c, s_ = math.cos(a), math.sin(a)
    fr = np.stack([c * f[0] - s_ * f[1], s_ * f[0] + c * f[1]])
    assert O.energy(BEC, BEC_PRM, fr, dx, dx) == pytest.approx(O.energy(BEC, BEC_PRM, f, dx, dx), rel=1e-13)
    Gf, Gr = O.force(BEC, BEC_PRM, f, dx, dx), O.force(BEC, BEC_PRM, fr, dx, dx)
    np.testing.assert_allclose(Gr, np.stack([c * Gf[0] - s_ * Gf[1], s_ * Gf[0] + c * Gf[1]]), rtol=0,
                               atol=1e-12 * np.abs(Gf).max())
    g90 = np.stack([_rot90_scalar(f[0]), _rot90_scalar(f[1])])
    assert O.energy(BEC, BEC_PRM, g90, dx, dx) == pytest.approx(O.energy(BEC, BEC_PRM, f, dx, dx), rel=1e-13)
    G90 = O.force(BEC, BEC_PRM, g90, dx, dx)
    np.testing.assert_allclose(G90, np.stack([_rot90_scalar(Gf[0]), _rot90_scalar(Gf[1])]), rtol=0,
                               atol=1e-11 * np.abs(Gf).max())
    # the rotation term is odd in Omega: the force changes under Omega -> -Omega
    assert np.abs(O.force(BEC, (1.3, -0.6, 2.0), f, dx, dx) - Gf).max() > 1e-3 * np.abs(Gf).max()


def _bec_ground_state(g, mu):
    """Radial Gross-Pitaevskii ground state at chemical potential mu (Omega = 0):
    -f''/2 - f'/(2r) + r^2 f/2 + g f^3 = mu f, f'(0) = 0, f -> 0; shooting on f(0)."""
    from scipy.integrate import quad, solve_ivp

    def rhs(r, y):
        f, fp = y
        return [fp, -fp / r + (r * r + 2 * g * f * f - 2 * mu) * f]

    def shoot(f0):
        r0 = 1e-6
        c = (2 * g * f0 ** 3 - 2 * mu * f0) / 4
        return solve_ivp(rhs, (r0, 10.0), [f0 + c * r0 * r0, 2 * c * r0], rtol=1e-12, atol=1e-14,
                         dense_output=True, events=[lambda r, y: y[0], lambda r, y: y[1]])

    lo, hi = 0.1, 1.5 * math.sqrt(mu / g)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if shoot(mid).t_events[0].size:
            lo = mid  # crosses zero: f(0) too small
        else:
            hi = mid
    sol = shoot(lo)
    rs = np.linspace(1e-6, sol.t[-1], 40000)
    rc = rs[np.argmin(np.abs(sol.sol(rs)[0]))]

    def edens(r):
        f, fp = sol.sol(r)
        return r * (0.5 * fp * fp + 0.5 * r * r * f * f + 0.5 * g * f ** 4 - mu * f * f)

    E = 2 * math.pi * quad(edens, 1e-6, rc, limit=500)[0]
    N = 2 * math.pi * quad(lambda r: r * sol.sol(r)[0] ** 2, 1e-6, rc, limit=500)[0]
    return E, N, lo


@pytest.mark.slow
def test_bec_ground_state_is_the_radial_solution_and_near_thomas_fermi():
    """Omega = 0: the arrested flow from the Thomas-Fermi ansatz relaxes to the radial
    Gross-Pitaevskii ground state (independent shooting solution), its energy at fourth
    order in dx; at mu = 10 the density is close to the Thomas-Fermi profile
    (mu - r^2/2)/g: N within 2% of pi mu^2 / g and the centre density within 1% of mu/g."""
    g, mu = 1.0, 10.0
    E, N, f0 = _bec_ground_state(g, mu)
    assert abs(N / (math.pi * mu * mu / g) - 1) < 0.02
    assert abs(f0 * f0 / (mu / g) - 1) < 0.01
    errs = []
    for n, dx in ((81, 0.2), (161, 0.1)):
        f = O.ansatz_bec((g, 0.0, mu), [], n, n, dx, dx)
        r = O.minimise(BEC, (g, 0.0, mu), f, dx, dx, tol=1e-7, max_steps=20000)
        assert r["converged"]
        o = O.observables(BEC, (g, 0.0, mu), r["f"], dx, dx)
        errs.append(abs(o["energy"] - E))
        assert o["atoms"] == pytest.approx(N, rel=1e-5)
        assert o["angular_momentum"] == pytest.approx(0.0, abs=1e-8)
        c = n // 2
        assert r["f"][0, c, c] ** 2 + r["f"][1, c, c] ** 2 == pytest.approx(f0 * f0, rel=1e-4)
    assert errs[1] < 1e-6 * abs(E)
    assert 12.0 < errs[0] / errs[1] < 20.0


# ---------------------------------------------------------------- BEC at a fixed atom number
def _zero_halo(f):
    f = f.copy()
    f[:, :2, :] = 0.0
    f[:, -2:, :] = 0.0
    f[:, :, :2] = 0.0
    f[:, :, -2:] = 0.0
    return f


def test_bec_fixed_n_refresh_scales_projects_and_takes_the_multiplier():
    """The refresh of a new field: N_h exactly N0; v tangent to the constraint
    (sum_I v.psi = 0); the halo untouched; the force at the multiplier orthogonal to
    psi; and, with a zero halo (so every stencil sees s psi), the multiplier of the
    scaled field in closed form (sum_I G_lin.psi + 2 g s^2 sum_I |psi|^4) / (2 sum_I |psi|^2),
    G_lin the force at g = 0 and mu = 0 of the unscaled field."""
    nx, ny, dx, dy = 41, 37, 0.21, 0.19
    g, Om, N0 = 1.3, 0.4, 7.5
    f = _zero_halo(I.smooth_field(BEC, nx, ny, dx, dy, seed=71))
    v = I.smooth_velocity(BEC, nx, ny, dx, dy, seed=72, amplitude=0.3)
    fr, vr, mu = O.bec_refresh((g, Om), N0, f, v, dx, dy)
    In = (slice(None), slice(2, -2), slice(2, -2))
    assert dx * dy * (fr[In] ** 2).sum() == pytest.approx(N0, rel=1e-14)
    assert abs((vr * fr).sum()) <= 1e-13 * (np.abs(vr) * np.abs(fr)).sum()
    ring = np.ones((ny, nx), bool)
    ring[2:-2, 2:-2] = False
    v[:, 2, 5] = 0.7  # a velocity on the first interior row changes; the halo's does not
    v[:, 0, 3] = 0.2
    fr, vr, mu = O.bec_refresh((g, Om), N0, f, v, dx, dy)
    assert np.array_equal(vr[:, ring], v[:, ring]) and vr[0, 2, 5] != 0.7
    G = O.force(BEC, (g, Om, mu), fr, dx, dy)
    assert abs((G * fr).sum()) <= 1e-12 * (np.abs(G) * np.abs(fr)).sum()
    S = (f[In] ** 2).sum()
    sc = math.sqrt(N0 / (dx * dy * S))
    assert np.abs(fr - sc * f).max() <= 1e-15 * sc * np.abs(f).max()
    A = (O.force(BEC, (0.0, Om, 0.0), f, dx, dy) * f).sum()
    B = ((f[0] ** 2 + f[1] ** 2) ** 2)[2:-2, 2:-2].sum()
    assert mu == pytest.approx((A + 2 * g * sc * sc * B) / (2 * S), rel=1e-12)
    # a field with a non-zero halo keeps it
    h = I.smooth_field(BEC, nx, ny, dx, dy, seed=73)
    hr, _, _ = O.bec_refresh((g, Om), N0, h, None, dx, dy)
    assert np.array_equal(hr[:, ring], h[:, ring])
    with pytest.raises(ValueError):
        O.bec_refresh((g, Om), N0, np.zeros_like(f), None, dx, dy)


def _bec_gc(g, mu, n, dx):
    f = O.ansatz_bec((g, 0.0, mu), [], n, n, dx, dx)
    r = O.minimise(BEC, (g, 0.0, mu), f, dx, dx, tol=1e-9, max_steps=40000)
    assert r["converged"]
    return r, O.observables(BEC, (g, 0.0, mu), r["f"], dx, dx)


@pytest.mark.parametrize("start", ["thomas_fermi", "smooth"])
def test_bec_fixed_n_relaxes_to_the_grand_canonical_ground_state(start):
    """The canonical problem at N = N_h of the grand-canonical ground state at mu (Omega
    = 0) has that ground state as its solution: the fixed-N flow from another start
    (a Thomas-Fermi profile at a different mu, or a smooth random complex field; zero
    halo in both) ends on the same density (the phase is free), with multiplier mu and
    energy E_gc + mu N; gradient descent at fixed N likewise."""
    g, mu, n, dx = 1.0, 4.0, 49, 0.2
    r, o = _bec_gc(g, mu, n, dx)
    N = o["atoms"]
    rho = r["f"][0] ** 2 + r["f"][1] ** 2
    if start == "thomas_fermi":
        f0 = O.ansatz_bec((g, 0.0, 2.5), [], n, n, dx, dx)
    else:
        f0 = _zero_halo(I.smooth_field(BEC, n, n, dx, dx, seed=5))
    for res in (O.minimise_fixed_n((g, 0.0), N, f0, dx, dx, 1e-9, 40000),
                O.gd_minimise_fixed_n((g, 0.0), N, f0, dx, dx, 1e-9, 200000)):
        assert res["converged"]
        rf = res["f"]
        assert np.abs(rf[0] ** 2 + rf[1] ** 2 - rho).max() < 1e-7 * rho.max()
        assert res["mu"] == pytest.approx(mu, abs=1e-7)
        assert res["energy"] == pytest.approx(o["energy"] + mu * N, rel=1e-10)
        assert dx * dx * (rf[:, 2:-2, 2:-2] ** 2).sum() == pytest.approx(N, rel=1e-14)


def test_bec_fixed_n_multiplier_is_dE_dN():
    """The multiplier is the chemical potential of the canonical ground state: the
    central difference of E(N) at N (1 +- 1e-3) against the multiplier at N."""
    g, n, dx, N = 1.0, 49, 0.2, 40.0
    f0 = O.ansatz_bec((g, 0.0, math.sqrt(g * N / math.pi)), [], n, n, dx, dx)
    E = {}
    for s in (0.999, 1.0, 1.001):
        res = O.minimise_fixed_n((g, 0.0), N * s, f0, dx, dx, 1e-10, 40000)
        assert res["converged"]
        E[s] = res
    dEdN = (E[1.001]["energy"] - E[0.999]["energy"]) / (0.002 * N)
    assert dEdN == pytest.approx(E[1.0]["mu"], rel=2e-5)
    # and the Thomas-Fermi value sqrt(g N / pi) is close (the kinetic term is small)
    assert E[1.0]["mu"] == pytest.approx(math.sqrt(g * N / math.pi), rel=0.05)


# ---------------------------------------------------------------- s+id superconductor (Table 1)
@pytest.mark.parametrize("nu", [0.0, 0.35])
def test_sid_reduces_to_abelian_higgs_without_the_d_band(nu):
    """Delta_d = 0: the s+id functional is the Abelian Higgs one with
    lambda/8 (u^2 - |psi|^2)^2 = a1 |psi|^2 + b1 |psi|^4 + lambda u^4 / 8 (a1 = -lambda u^2 / 4,
    b1 = lambda / 8), so E_h differs by area(I) lambda u^4 / 8 and the forces on Delta_s and
    A are the Abelian Higgs ones; the d band feels a force only through the mixed
    gradient (nu != 0)."""
    nx, ny, dx, dy = 30, 26, 0.3, 0.25
    lam, u = 1.4, 1.1
    ah = I.smooth_field(AH, nx, ny, dx, dy, seed=31)
    f = np.zeros((6, ny, nx))
    f[0], f[1], f[4], f[5] = ah[0], ah[1], ah[2], ah[3]
    prm = (-lam * u * u / 4, -0.6, lam / 8, 0.4, 0.3, 0.15, nu)
    area = (nx - 4) * (ny - 4) * dx * dy
    assert O.energy(SID, prm, f, dx, dy) == pytest.approx(O.energy(AH, (lam, u), ah, dx, dy) - area * lam * u ** 4 / 8,
                                                         rel=1e-13)
    G, Ga = O.force(SID, prm, f, dx, dy), O.force(AH, (lam, u), ah, dx, dy)
    sc = np.abs(Ga).max()
    for c, ca in ((0, 0), (1, 1), (4, 2), (5, 3)):
        np.testing.assert_allclose(G[c], Ga[ca], rtol=0, atol=1e-12 * sc)
    if nu == 0.0:
        assert not G[2].any() and not G[3].any()
    else:
        assert np.abs(G[2:4]).max() > 1e-3 * sc


def test_sid_d_wave_rotation_and_band_symmetries():
    """The mixed gradient nu (|D_1 . |^2-type with eta = (1, -1)) has d_{x^2-y^2} symmetry: a
    90-degree rotation of space and A together with Delta_d -> -Delta_d leaves E_h exactly
    invariant (without the sign flip it does not, for nu != 0). Exchanging the bands with
    their couplings (a1 <-> a2, b1 <-> b2) is exact too."""
    n, dx = 26, 0.3
    f = I.smooth_field(SID, n, n, dx, dx, seed=41)
    r = _rot90_scalar
    E0 = O.energy(SID, SID_PRM, f, dx, dx)
    g = np.stack([r(f[0]), r(f[1]), -r(f[2]), -r(f[3]), -r(f[5]), r(f[4])])
    assert O.energy(SID, SID_PRM, g, dx, dx) == pytest.approx(E0, rel=1e-13)
    g2 = g.copy()
    g2[2:4] *= -1
    assert abs(O.energy(SID, SID_PRM, g2, dx, dx) - E0) > 1e-4 * abs(E0)
    Gf, Gg = O.force(SID, SID_PRM, f, dx, dx), O.force(SID, SID_PRM, g, dx, dx)
    Grot = np.stack([r(Gf[0]), r(Gf[1]), -r(Gf[2]), -r(Gf[3]), -r(Gf[5]), r(Gf[4])])
    np.testing.assert_allclose(Gg, Grot, rtol=0, atol=1e-11 * np.abs(Gf).max())
    a1, a2, b1, b2, b3, b4, nu = SID_PRM
    sw = np.stack([f[2], f[3], f[0], f[1], f[4], f[5]])
    assert O.energy(SID, (a2, a1, b2, b1, b3, b4, nu), sw, dx, dx) == pytest.approx(E0, rel=1e-13)


def test_sid_gauge_invariance_fourth_order():
    """Delta_a -> e^{i chi} Delta_a, A -> A + grad chi: E_h changes at O(h^4)."""
    errs = []
    for n in (41, 81):
        L = 8.0
        dx = L / (n - 1)
        dy = 0.9 * dx
        X, Y = grid(n, n, dx, dy)
        f = I.smooth_field(SID, n, n, dx, dy, seed=6)
        chi = 0.7 * np.sin(0.5 * X + 0.2) * np.cos(0.6 * Y) + 0.1 * X * Y
        cx = 0.35 * np.cos(0.5 * X + 0.2) * np.cos(0.6 * Y) + 0.1 * Y
        cy = -0.42 * np.sin(0.5 * X + 0.2) * np.sin(0.6 * Y) + 0.1 * X
        c, s_ = np.cos(chi), np.sin(chi)
        g = np.stack([c * f[0] - s_ * f[1], s_ * f[0] + c * f[1], c * f[2] - s_ * f[3], s_ * f[2] + c * f[3],
                      f[4] + cx, f[5] + cy])
        errs.append(abs(O.energy(SID, SID_PRM, g, dx, dy) - O.energy(SID, SID_PRM, f, dx, dy)))
    assert errs[0] / errs[1] > 12.0 and errs[1] < 2e-4


def test_sid_uniform_ground_state_closed_form():
    """Uniform fields: only the potential survives. For b4 > 0 the relative phase pi/2
    (s + i d) minimises it, and a1 + 2 b1 S + (b3 - 2 b4) D = a2 + 2 b2 D + (b3 - 2 b4) S = 0
    fixes S = |Delta_s|^2, D = |Delta_d|^2 (here S = 1, D = 0.75): the force vanishes there
    and E_h is area(I) times the potential's minimum; a relative phase 0 raises it."""
    a1, a2, b1, b2, b3, b4, nu = SID_PRM
    b3e = b3 - 2 * b4
    S, D = np.linalg.solve([[2 * b1, b3e], [b3e, 2 * b2]], [-a1, -a2])
    assert S == pytest.approx(1.0) and D == pytest.approx(0.75)
    assert O.ansatz_sid(SID_PRM, [[0, 0, 0, 1.0, 0]], 8, 8, 0.3, 0.3)[1] == pytest.approx((S, D, math.pi / 2))
    nx, ny, dx, dy = 14, 12, 0.3, 0.2
    f = np.zeros((6, ny, nx))
    f[0] = math.sqrt(S)
    f[3] = math.sqrt(D)  # Delta_d = i sqrt(D): relative phase pi/2
    area = (nx - 4) * (ny - 4) * dx * dy
    Vmin = a1 * S + a2 * D + b1 * S * S + b2 * D * D + b3e * S * D
    assert O.energy(SID, SID_PRM, f, dx, dy) == pytest.approx(area * Vmin, rel=1e-13)
    assert np.abs(O.force(SID, SID_PRM, f, dx, dy)).max() < 1e-14
    g = f.copy()
    g[2], g[3] = math.sqrt(D), 0.0  # relative phase 0
    assert O.energy(SID, SID_PRM, g, dx, dy) > O.energy(SID, SID_PRM, f, dx, dy) + area * 4 * b4 * S * D * 0.99


# ---------------------------------------------------------------- demagnetisation (Eq. 6)
def test_demag_energy_of_a_single_mode_is_the_discrete_closed_form():
    """n_1 = a cos(k x') sin(q y'), measured from the zero boundary nodes next to I
    (x' = (i - 1) dx), with k, q fitting the box: the Eq. 1 divergence is the pure mode
    -a s1 sin(k x') sin(q y') (s1 the Eq. 1 symbol), the 5-point Laplacian multiplies it by
    lambda = -(2 - 2 cos k dx)/dx^2 - (2 - 2 cos q dy)/dy^2, so
    E_ms = -mu_d/2 dx dy sum_I rho^2 / lambda exactly."""
    nx, ny, dx, dy = 30, 24, 0.3, 0.25
    X, Y = np.meshgrid((np.arange(nx) - 1) * dx, (np.arange(ny) - 1) * dy)
    Lx, Ly = (nx - 3) * dx, (ny - 3) * dy
    a, k, q = 0.4, 2 * math.pi / Lx, math.pi / Ly
    f = np.zeros((3, ny, nx))
    f[0] = a * np.cos(k * X) * np.sin(q * Y)
    s1 = (8 * math.sin(k * dx) - math.sin(2 * k * dx)) / (6 * dx)
    lam = -(2 - 2 * math.cos(k * dx)) / dx ** 2 - (2 - 2 * math.cos(q * dy)) / dy ** 2
    rho = -a * s1 * np.sin(k * X) * np.sin(q * Y)
    sl = (slice(2, ny - 2), slice(2, nx - 2))
    exp = -0.5 * CMD_PRM[5] * dx * dy * (rho[sl] ** 2).sum() / lam
    assert O.demag_energy(CMD_PRM, f, dx, dy) == pytest.approx(exp, rel=1e-13)
    r, psi = O.demag_potential(f, dx, dy)
    np.testing.assert_allclose(r[sl], rho[sl], rtol=0, atol=1e-14)
    np.testing.assert_allclose(psi[sl], rho[sl] / lam, rtol=0, atol=1e-14)


def test_demag_potential_solves_the_five_point_poisson_problem():
    """On a general field the sine-transform solution satisfies the 5-point stencil
    equation L psi = rho on I directly, with psi = 0 on the halo, and E_ms > 0."""
    nx, ny, dx, dy = 33, 27, 0.3, 0.25
    f = I.smooth_field(CM, nx, ny, dx, dy, seed=19)
    rho, psi = O.demag_potential(f, dx, dy)
    sl = (slice(2, ny - 2), slice(2, nx - 2))
    L = np.zeros_like(psi)
    L[1:-1, 1:-1] = ((psi[1:-1, 2:] - 2 * psi[1:-1, 1:-1] + psi[1:-1, :-2]) / dx ** 2 +
                     (psi[2:, 1:-1] - 2 * psi[1:-1, 1:-1] + psi[:-2, 1:-1]) / dy ** 2)
    np.testing.assert_allclose(L[sl], rho[sl], rtol=0, atol=1e-12 * np.abs(rho).max())
    assert not psi[:2].any() and not psi[-2:].any() and not psi[:, :2].any() and not psi[:, -2:].any()
    assert O.demag_energy(CMD_PRM, f, dx, dy) > 0.0
    assert O.energy(CMD, CMD_PRM, f, dx, dy) == pytest.approx(
        O.energy(CM, CMD_PRM[:5], f, dx, dy) + O.demag_energy(CMD_PRM, f, dx, dy), rel=1e-14)


def test_demag_box_is_the_smallest_fft_friendly_one():
    """The Dirichlet box along an axis of N sites: N' + 1 has no prime factor above 7,
    no smaller N' >= N has that property, and floor((N' - N) / 2) sites go below I."""
    def smooth(m):
        for q in (2, 3, 5, 7):
            while m % q == 0:
                m //= q
        return m == 1
    for N in list(range(1, 300)) + [1020, 2044, 4092, 8188]:
        Np, below = O.demag_box(N)
        assert Np >= N and smooth(Np + 1) and not any(smooth(m + 1) for m in range(N, Np))
        assert below == (Np - N) // 2
    assert O.demag_box(4092) == (4095, 1)  # 4093 is prime: the box adds 3 sites


def test_demag_padded_box_solves_the_five_point_poisson_problem():
    """A grid whose interior needs padding (60 and 36 sites: 61 and 37 are prime): the
    box potential satisfies L psi = rho on every box site, with rho the charge on I and
    zero on the padding, vanishes on the box's outer nodes, and the stored potential is
    the box solution on I and zero on the halo."""
    nx, ny, dx, dy = 64, 40, 0.3, 0.25
    (Nx, bx), (Ny, by) = O.demag_box(nx - 4), O.demag_box(ny - 4)
    assert (Nx, bx, Ny, by) == (62, 1, 39, 1)
    f = I.smooth_field(CM, nx, ny, dx, dy, seed=23)
    rho, psi = O.demag_potential(f, dx, dy)
    box = O.demag_box_potential(f, dx, dy)
    assert box.shape == (Ny + 2, Nx + 2)
    assert not box[0].any() and not box[-1].any() and not box[:, 0].any() and not box[:, -1].any()
    rb = np.zeros_like(box)
    rb[1 + by:1 + by + ny - 4, 1 + bx:1 + bx + nx - 4] = rho[2:-2, 2:-2]
    L = ((box[1:-1, 2:] - 2 * box[1:-1, 1:-1] + box[1:-1, :-2]) / dx ** 2 +
         (box[2:, 1:-1] - 2 * box[1:-1, 1:-1] + box[:-2, 1:-1]) / dy ** 2)
    np.testing.assert_allclose(L, rb[1:-1, 1:-1], rtol=0, atol=1e-12 * np.abs(rho).max())
    assert np.array_equal(psi[2:-2, 2:-2], box[1 + by:1 + by + ny - 4, 1 + bx:1 + bx + nx - 4])
    assert not psi[:2].any() and not psi[-2:].any() and not psi[:, :2].any() and not psi[:, -2:].any()
    assert np.abs(box[1:-1, 1:-1]).max() > 0 and abs(box[1 + by, 1]) > 0  # the padding carries potential


def test_demag_gradient_is_exact_on_a_padded_box():
    """Brute-force lattice gradient of the full energy with demagnetisation where the
    Dirichlet box is larger than I (both axes padded): the force uses psi on I only,
    which is the exact gradient of -mu_d/2 dx dy sum_I psi rho for any box."""
    nx, ny, dx, dy = 14, 40, 0.3, 0.25
    assert O.demag_box(nx - 4) == (11, 0) and O.demag_box(ny - 4) == (39, 1)  # padded above; below and above
    f = I.smooth_field(CMD, nx, ny, dx, dy, seed=29, amplitude=0.5)
    grad = O.energy_grad_exact(CMD, CMD_PRM, f, dx, dy)
    eps = 1e-6
    fd = np.zeros_like(f)
    for idx in np.ndindex(f.shape):
        fp, fm = f.copy(), f.copy()
        fp[idx] += eps
        fm[idx] -= eps
        fd[idx] = (O.energy(CMD, CMD_PRM, fp, dx, dy) - O.energy(CMD, CMD_PRM, fm, dx, dy)) / (2 * eps)
    np.testing.assert_allclose(grad, fd, rtol=0, atol=1e-7 * np.abs(grad).max())


def test_demag_spares_bloch_and_charges_neel_skyrmions():
    """The magnetostatic energy comes from the in-plane divergence: a Bloch skyrmion
    (helicity pi/2, divergence-free) has none beyond the stencils' O(h^4) remainder,
    a Neel one (helicity 0, radial in-plane part) a finite amount."""
    e = {}
    for n in (61, 121):
        d = 16.0 / (n - 1)
        X, Y = grid(n, n, d, d)
        fr = np.pi * np.exp(-(np.hypot(X, Y) / 2.0) ** 2)
        for gam in (0.0, np.pi / 2):
            th = np.arctan2(Y, X) + gam
            ff = np.stack([np.sin(fr) * np.cos(th), np.sin(fr) * np.sin(th), np.cos(fr)])
            e[(n, gam)] = O.demag_energy(CMD_PRM, ff, d, d)
    assert e[(121, 0.0)] == pytest.approx(e[(61, 0.0)], rel=1e-2) and e[(121, 0.0)] > 1.0
    assert e[(61, np.pi / 2)] < 1e-6 * e[(61, 0.0)] and e[(121, np.pi / 2)] < 1e-2 * e[(61, np.pi / 2)]


# ---------------------------------------------------------------- force (Eq. 3's right-hand side)
def _prm(theory):
    return {AH: AH_PRM, CM: (1.0, 0.8, 0.15, 0.5, 0.0), BS: BS_PRM, BEC: BEC_PRM, SID: SID_PRM, CMD: CMD_PRM}[theory]


@pytest.mark.parametrize("theory", [AH, CM, BS, BEC, SID, CMD])
def test_exact_gradient_matches_brute_force(theory):
    nx, ny, dx, dy = 12, 11, 0.3, 0.25
    prm = _prm(theory)
    f = I.smooth_field(theory, nx, ny, dx, dy, seed=21, amplitude=0.5)
    grad = O.energy_grad_exact(theory, prm, f, dx, dy)
    eps = 1e-6
    fd = np.zeros_like(f)
    for idx in np.ndindex(f.shape):
        fp, fm = f.copy(), f.copy()
        fp[idx] += eps
        fm[idx] -= eps
        fd[idx] = (O.energy(theory, prm, fp, dx, dy) - O.energy(theory, prm, fm, dx, dy)) / (2 * eps)
    np.testing.assert_allclose(grad, fd, rtol=0, atol=1e-7 * np.abs(grad).max())


@pytest.mark.parametrize("theory", [AH, CM, BS, BEC, SID, CMD])
def test_force_is_energy_gradient_to_fourth_order(theory):
    """dx dy G and dE_h/dphi (tangent part for the unit-vector theories) are two O(h^4)
    discretisations of the same Euler-Lagrange expression: their gap shrinks ~16x per halving."""
    prm = _prm(theory)
    errs = []
    for n in (41, 81):
        L = 8.0
        dx = L / (n - 1)
        dy = 0.9 * dx
        # the quartic Skyrme term needs a gentler field to be in the asymptotic regime
        f = I.smooth_field(theory, n, n, dx, dy, seed=7, amplitude=0.15 if theory == BS else 0.3)
        G = O.force(theory, prm, f, dx, dy)
        gr = O.energy_grad_exact(theory, prm, f, dx, dy) / (dx * dy)
        if theory in (CM, BS, CMD):
            gr = gr - (gr * f).sum(axis=0, keepdims=True) * f
        k = 4 if n == 41 else 8  # same physical margin on both grids
        errs.append(np.abs(G - gr)[:, k:-k, k:-k].max() / np.abs(G).max())
    assert errs[0] / errs[1] > 12.0, errs
    assert errs[1] < 5e-3


# ---------------------------------------------------------------- time integrator (Eq. 3, Eq. 4)
def _rk4_matrix(omega2, dt):
    """Classic RK4 on y' = M y is the degree-4 Taylor polynomial of exp(dt M)."""
    M = np.array([[0.0, 1.0], [-omega2, 0.0]])
    Z = dt * M
    return np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24


def test_rk4_and_arrest_on_harmonic_oscillator():
    """Harmonic test field (e = k phi^2 / 2 on the single interior site of a 5x5 grid):
    every step must equal the closed-form RK4 propagator, and the velocity must be
    zeroed exactly on the steps where the energy rises (Eq. 4)."""
    k, dt = 4.0, 0.3
    T = _rk4_matrix(k, dt)
    f = np.zeros((1, 5, 5))
    v = np.zeros((1, 5, 5))
    f[0, 2, 2] = 1.0
    E = 0.5 * k
    y = np.array([1.0, 0.0])
    Eref = 0.5 * k
    n_arrest = 0
    for _ in range(120):
        f, v, E, arrested = O.anf_step(HARM, (k,), f, v, 1.0, 1.0, dt, E)
        y = T @ y
        Enew = 0.5 * k * y[0] ** 2
        exp_arrest = Enew > Eref
        if exp_arrest:
            y[1] = 0.0
        Eref = Enew
        assert arrested == exp_arrest
        n_arrest += arrested
        assert f[0, 2, 2] == pytest.approx(y[0], abs=1e-13)
        assert v[0, 2, 2] == pytest.approx(y[1], abs=1e-13)
        assert E == pytest.approx(Enew, abs=1e-13)
        # halo untouched
        assert np.count_nonzero(f) <= 1 and np.count_nonzero(v) <= 1
    assert n_arrest >= 1
    assert abs(f[0, 2, 2]) < 1e-2  # arrested flow has relaxed the oscillator


def test_minimise_stops_at_tolerance():
    k, dt = 4.0, 0.3
    f = np.zeros((1, 5, 5))
    f[0, 2, 2] = 1.0
    r = O.minimise(HARM, (k,), f, 1.0, 1.0, tol=1e-9, max_steps=10_000, dt=dt)
    assert r["converged"] and abs(k * r["f"][0, 2, 2]) < 1e-9
    r2 = O.minimise(HARM, (k,), f, 1.0, 1.0, tol=1e-9, max_steps=3, dt=dt)
    assert not r2["converged"] and r2["steps"] == 3


def test_cm_flow_keeps_unit_length():
    p = I.cm_skyrmions(n=96, count=2, seed=3, min_sep=8.0, margin=4.0)
    f = O.ansatz(CM, p.soliton_array(), p.nx, p.ny, p.dx, p.dy)
    v = np.zeros_like(f)
    E = O.energy(CM, p.params, f, p.dx, p.dy)
    dt = O.time_step(p.dx, p.dy)
    for _ in range(20):
        f, v, E, _ = O.anf_step(CM, p.params, f, v, p.dx, p.dy, dt, E)
    assert np.abs(np.sqrt((f * f).sum(axis=0)) - 1.0).max() < 1e-14
    assert np.abs((f * v).sum(axis=0)).max() < 1e-14  # velocity stays tangent
    assert O.observables(CM, p.params, f, p.dx, p.dy)["charge"] == pytest.approx(-2.0, abs=1e-10)


# ---------------------------------------------------------------- gradient descent (Sec. 3.2's first-order alternative)
def test_gd_on_harmonic_field_is_the_closed_form_geometric_decay():
    """e = k phi^2 / 2 on one interior site: each step multiplies phi by (1 - dtau k)
    exactly; the energy rises on every step once |1 - dtau k| > 1, never before; the
    minimiser stops at the first n with dx dy k |phi_n| < tol."""
    k = 4.0
    for dtau, rising in ((0.1, False), (0.45, False), (0.55, True)):
        f = np.zeros((1, 5, 5))
        f[0, 2, 2] = 1.0
        E = 0.5 * k
        for n in range(1, 40):
            f, E, rose = O.gd_step(HARM, (k,), f, 1.0, 1.0, dtau, E)
            assert f[0, 2, 2] == pytest.approx((1.0 - dtau * k) ** n, rel=1e-13, abs=1e-300)
            assert E == pytest.approx(0.5 * k * (1.0 - dtau * k) ** (2 * n), rel=1e-12, abs=1e-300)
            assert rose == rising
            assert np.count_nonzero(f) == 1  # halo untouched
    f = np.zeros((1, 5, 5))
    f[0, 2, 2] = 1.0
    tol, dtau = 1e-9, 0.1
    r = O.gd_minimise(HARM, (k,), f, 1.0, 1.0, tol=tol, max_steps=10_000, dtau=dtau)
    n_exp = math.ceil(math.log(tol / k) / math.log(1.0 - dtau * k))
    assert r["converged"] and r["steps"] == n_exp and r["rises"] == 0
    r2 = O.gd_minimise(HARM, (k,), f, 1.0, 1.0, tol=tol, max_steps=5, dtau=dtau)
    assert not r2["converged"] and r2["steps"] == 5


@pytest.mark.parametrize("theory", [AH, CM])
def test_gd_step_descends_along_the_exact_gradient(theory):
    """d/dtau E_h(phi - dtau G) at 0 is -sum dE_h/dphi . G exactly (chain rule; the
    chiral-magnet renormalisation is second order since G is tangent). The exact
    gradient is pinned by brute force above, so this fixes the step's direction and
    scale; Richardson extrapolation in dtau removes the O(dtau) term."""
    nx, ny, dx, dy = 24, 21, 0.3, 0.25
    prm = AH_PRM if theory == AH else (1.0, 0.8, 0.15, 0.5, 0.0)
    f = I.smooth_field(theory, nx, ny, dx, dy, seed=5, amplitude=0.5)
    E0 = O.energy(theory, prm, f, dx, dy)
    G = O.force(theory, prm, f, dx, dy)
    slope = -(O.energy_grad_exact(theory, prm, f, dx, dy) * G).sum()
    d = []
    for t in (2e-5, 1e-5):
        _, E1, _ = O.gd_step(theory, prm, f, dx, dy, t, E0)
        d.append((E1 - E0) / t)
    rich = 2.0 * d[1] - d[0]
    assert slope < 0.0
    assert rich == pytest.approx(slope, rel=1e-6)


@pytest.mark.parametrize("theory", [AH, CM])
def test_gd_step_limit_is_sharp(theory):
    """Below the Eq. 2 stability limit the descent never raises the energy; just above
    it the checkerboard modes grow and the energy rises. Fixes the limit to a few %."""
    nx, ny, dx, dy = 40, 36, 0.3, 0.25
    prm = AH_PRM if theory == AH else (1.0, 0.8, 0.15, 0.5, 0.0)
    f = I.smooth_field(theory, nx, ny, dx, dy, seed=3, amplitude=0.3)
    rng = np.random.default_rng(1)
    f[:, 2:-2, 2:-2] += 1e-3 * rng.standard_normal(f[:, 2:-2, 2:-2].shape)
    if theory == CM:
        f[:, 2:-2, 2:-2] /= np.sqrt((f[:, 2:-2, 2:-2] ** 2).sum(axis=0))
    lim = O.gd_step_limit(dx, dy)
    assert lim == pytest.approx(3.0 / 8.0 / (1.0 / dx**2 + 1.0 / dy**2), rel=1e-15)
    rises = {}
    for s in (0.95, 1.02):
        g, E, n = f.copy(), O.energy(theory, prm, f, dx, dy), 0
        for _ in range(300):
            g, E, r = O.gd_step(theory, prm, g, dx, dy, s * lim, E)
            n += r
        rises[s] = n
    assert rises[0.95] == 0 and rises[1.02] > 50
    if theory == CM:
        assert np.abs(np.sqrt((g * g).sum(axis=0)) - 1.0).max() < 1e-14


def test_gd_and_arrested_flow_reach_the_same_vortex():
    """Both minimisers stop at a stationary point of the same E_h: for one centred
    vortex (a unique minimum) the energies agree far below the lattice error."""
    n, dx = 48, 0.25
    f = O.ansatz(AH, [[0.0, 0.0, 1.0, 1.0, 0.0]], n, n, dx, dx)
    a = O.minimise(AH, AH_PRM, f, dx, dx, tol=1e-6, max_steps=20_000)
    g = O.gd_minimise(AH, AH_PRM, f, dx, dx, tol=1e-6, max_steps=100_000)
    assert a["converged"] and g["converged"] and g["rises"] == 0
    assert abs(a["energy"] - g["energy"]) < 1e-8 * a["energy"]
    assert np.abs(a["f"] - g["f"]).max() < 1e-4  # ~ tol / lowest Hessian eigenvalue
    assert g["steps"] > a["steps"]  # the first-order flow needs more (cheaper) steps


# ---------------------------------------------------------------- observables and physics
def test_berg_luescher_charge_is_exact_integer():
    n, dx = 96, 0.2
    sol = [[-5.0, -4.0, 1.0, 2.0, 0.0], [4.0, 3.0, 1.0, 2.5, 1.0], [-3.0, 5.0, -1.0, 2.0, 0.0]]
    f = O.ansatz(CM, sol, n, n, dx, dx)
    assert O.observables(CM, CM_PRM, f, dx, dx)["charge"] == pytest.approx(-1.0 - 1.0 + 1.0, abs=1e-12)
    f1 = O.ansatz(CM, sol[:1], n, n, dx, dx)
    assert O.observables(CM, CM_PRM, f1, dx, dx)["charge"] == pytest.approx(-1.0, abs=1e-12)


def test_ah_winding_and_flux_of_ansatz():
    n, dx = 128, 0.125
    g = golden()["flux_per_unit_winding"]["value_over_pi"]
    for sol in ([[0.0, 0.0, 1.0, 1.0, 0.0]],
                [[-1.0, 0.5, 1.0, 1.0, 0.0], [1.2, -0.7, 1.0, 1.0, 0.3]],
                [[-1.0, 0.0, 1.0, 1.0, 0.0], [1.0, 1.0, 1.0, 1.0, 0.0], [0.2, -1.3, 1.0, 1.0, 0.0]]):
        N = len(sol)
        o = O.observables(AH, AH_PRM, O.ansatz(AH, sol, n, n, dx, dx), dx, dx)
        assert o["charge"] == pytest.approx(N, abs=1e-12)
        assert o["flux"] == pytest.approx(g * math.pi * N, rel=2e-3)


@pytest.mark.slow
@pytest.mark.parametrize("N", [1, 2])
def test_ah_relaxes_to_bogomolny_bound(N):
    """At lambda = 1 the relaxed N-vortex energy sits at pi N (Bogomolny bound of Table 1's
    functional), the flux at 2 pi N and the winding at N."""
    g = golden()
    n, dx = 64, 0.2
    f = O.ansatz(AH, [[0.0, 0.0, float(N), 1.0, 0.0]], n, n, dx, dx)
    r = O.minimise(AH, AH_PRM, f, dx, dx, tol=1e-6, max_steps=5000)
    assert r["converged"]
    o = O.observables(AH, AH_PRM, r["f"], dx, dx)
    bound = g["bogomolny_energy_per_unit_winding"]["value_over_pi"] * math.pi * N
    assert abs(o["energy"] - bound) < 3e-4 * bound  # lattice error at dx = 0.2
    assert o["flux"] == pytest.approx(g["flux_per_unit_winding"]["value_over_pi"] * math.pi * N, rel=5e-3)
    assert o["charge"] == pytest.approx(N, abs=1e-12)


@pytest.mark.slow
def test_ah_energy_ordering_with_coupling():
    """Away from critical coupling a single vortex lies below pi for lambda < 1 and above for lambda > 1."""
    n, dx = 64, 0.2
    f = O.ansatz(AH, [[0.0, 0.0, 1.0, 1.0, 0.0]], n, n, dx, dx)
    e = {}
    for lam in (0.5, 2.0):
        r = O.minimise(AH, (lam, 1.0), f, dx, dx, tol=1e-6, max_steps=8000)
        assert r["converged"]
        e[lam] = r["energy"]
    assert e[0.5] < math.pi - 0.05 < math.pi + 0.05 < e[2.0]


# ---------------------------------------------------------------- input generator
def test_splitmix64_reference_value():
    # first output of SplitMix64 seeded with 0 (published reference sequence)
    assert I.SplitMix64(0).next_u64() == 0xE220A8397B1DCDAF


def test_workload_generators_are_deterministic_and_valid():
    a = I.cm_skyrmions(n=1024, count=8)
    b = I.cm_skyrmions(n=1024, count=8)
    assert a.solitons == b.solitons
    pts = np.array([(s[0], s[1]) for s in a.solitons])
    d = np.hypot(pts[:, None, 0] - pts[None, :, 0], pts[:, None, 1] - pts[None, :, 1])
    assert (d[np.triu_indices(8, 1)] >= 8.0).all()
    half = 0.5 * 1023 * 0.2
    assert (np.abs(pts) <= half - 8.0).all()
    batch = I.ah_batch()
    assert len(batch) == 256
    assert {p.nx for p in batch} == {64, 128, 256, 512}
    for p in batch:
        L = p.nx * p.dx
        assert 0.5 <= p.params[0] < 2.0 and 1 <= len(p.solitons) <= 4
        assert all(abs(s[0]) <= L / 4 and abs(s[1]) <= L / 4 for s in p.solitons)
