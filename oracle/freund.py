"""Closed forms for the suddenly loaded crack of Sec. 5.2 (validation tools).

TEST INFRASTRUCTURE ONLY (part of the oracle package; see oracle/__init__.py).

* ``rayleigh_speed`` -- the surface-wave speed c_R, the root in (0, c_s) of
  (2 - c^2/c_s^2)^2 - 4 sqrt((1 - c^2/c_d^2)(1 - c^2/c_s^2)) = 0 (Sec. 5.2),
  and the approximation c_R ~ c_s (0.862 + 1.14 nu)/(1 + nu) quoted there.
* ``ki0`` -- K_I^0 = 2 t* sqrt(1 - 2 nu)/(1 - nu) sqrt(c_d t/pi), valid until the
  waves scattered by one tip reach the other (t < l_c/c_d).
* ``ki1`` -- K_I^1 of Eq. (ki1) for l_c/c_d < t < 2 l_c/c_d: K_I^0 plus a nested
  integral whose inner integrand has a pole at xi = eta and whose outer one has a
  pole at eta = c_r; both are Cauchy principal values (scipy's quad with the
  Cauchy weight).  Slownesses a = 1/c_d, b = 1/c_s, c_r = 1/c_R.

Reading of Eq. (ki1): the printed formula mixes a length (l_c) and slownesses;
it is dimensionally consistent with lengths in units of l_c and speeds in units
of c_d, so the integrals are evaluated with a = 1, b = c_d/c_s, c_r = c_d/c_R
and upper limit T = c_d t/l_c, and the correction is scaled by sqrt(l_c).
F_+(0) is the paper's value, 0.8774, stated for its material (nu = 0.2174);
its definition is not given, so other materials have no value of it here.
ki1: parity unpinned.  Its absolute level is pinned to nothing the paper fixes
(the figure is not available, and F_+(0) = 0.8774 does not follow from the
plain Wiener-Hopf factor, which gives 0.8085); the tests check continuity with
ki0 and compare it with the oracle's lattice run.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import quad
from scipy.optimize import brentq

F_PLUS_0_PAPER = 0.8774  # Sec. 5.2, for c_s^2/c_d^2 = 0.3611


def rayleigh_speed(cs: float, cd: float) -> float:
    """Rayleigh wave speed: the nonzero root in (0, c_s) of the equation of Sec. 5.2."""
    def r(c):
        x, y = (c / cs) ** 2, (c / cd) ** 2
        return (2.0 - x) ** 2 - 4.0 * math.sqrt((1.0 - y) * (1.0 - x))
    # r(0) = 0 is the trivial root; the surface wave lies in (0.5 c_s, c_s)
    return brentq(r, 0.5 * cs, cs * (1.0 - 1e-15), xtol=1e-15, rtol=1e-15)


def rayleigh_speed_approx(cs: float, nu: float) -> float:
    """The approximation c_R ~ c_s (0.862 + 1.14 nu)/(1 + nu) quoted in Sec. 5.2."""
    return cs * (0.862 + 1.14 * nu) / (1.0 + nu)


def ki0(t, tstar: float, nu: float, cd: float = 1.0):
    """K_I^0 of Sec. 5.2 (semi-infinite crack, valid for t < l_c/c_d)."""
    t = np.asarray(t, dtype=np.float64)
    return 2.0 * tstar * math.sqrt(1.0 - 2.0 * nu) / (1.0 - nu) * np.sqrt(cd * t / math.pi)


def ki_static(tstar: float, lc: float) -> float:
    """The quasistatic normalisation K_I^s = t* sqrt(pi l_c/2) of Sec. 5.2."""
    return tstar * math.sqrt(math.pi * lc / 2.0)


def _arg(xi: float, a: float, b: float) -> float:
    """arctan of 4 xi^2 sqrt((xi^2 - a^2)(b^2 - xi^2))/(b^2 - 2 xi^2)^2 (in [0, pi/2])."""
    num = 4.0 * xi * xi * math.sqrt(max(0.0, (xi * xi - a * a) * (b * b - xi * xi)))
    den = (b * b - 2.0 * xi * xi) ** 2
    return math.atan2(num, den)


def _inner(eta: float, a: float, b: float) -> float:
    """(1/pi) CPV int_a^b arctan(...) 2 eta/(xi^2 - eta^2) dxi  (the exponent of Eq. ki1)."""
    kink = b / math.sqrt(2.0)  # the arctan reaches pi/2 there
    pieces = [(a, kink), (kink, b)]
    total = 0.0
    for lo, hi in pieces:
        if lo < eta < hi:
            # CPV of g(xi)/(xi - eta), g = arctan(...) 2 eta/(xi + eta)
            val, _ = quad(lambda xi: _arg(xi, a, b) * 2.0 * eta / (xi + eta), lo, hi,
                          weight="cauchy", wvar=eta, limit=400)
        else:
            val, _ = quad(lambda xi: _arg(xi, a, b) * 2.0 * eta / (xi * xi - eta * eta), lo, hi,
                          limit=400)
        total += val
    return total / math.pi


def ki1(t, tstar: float, nu: float, cd: float, cs: float, lc: float,
        f_plus_0: float = F_PLUS_0_PAPER):
    """K_I^1 of Eq. (ki1) for l_c/c_d <= t <= 2 l_c/c_d (K_I^0 for earlier t)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    a, b = 1.0, cd / cs
    cr = cd / rayleigh_speed(cs, cd)
    out = np.empty_like(t)
    for n, tt in enumerate(t):
        k0 = float(ki0(tt, tstar, nu, cd))
        T = cd * tt / lc
        if T <= a:
            out[n] = k0
            continue

        def g(eta):
            # Im of sqrt(T - eta) sqrt((a - eta)/(a + eta)) (c_r + eta)/(c_r - eta) exp(J)/eta
            # without the pole factor 1/(c_r - eta); sqrt of the negative ratio is +i sqrt(.)
            return (math.sqrt(max(0.0, T - eta)) * math.sqrt(max(0.0, (eta - a) / (eta + a))) *
                    (cr + eta) * math.exp(_inner(eta, a, b)) / eta)

        if T > cr * (1.0 + 1e-9):
            # CPV of g/(c_r - eta) = -g/(eta - c_r) over [a, T]
            v1, _ = quad(lambda e: -g(e), a, T, weight="cauchy", wvar=cr, limit=400)
            val = v1
        else:
            val, _ = quad(lambda e: g(e) / (cr - e), a, T, limit=400)
        corr = 2.0 * tstar * f_plus_0 / math.pi * math.sqrt(2.0 / math.pi) * val
        out[n] = k0 + corr * math.sqrt(lc)
    return out if out.size > 1 else float(out[0])
