"""Oracle pins: dynamics against conservation laws and closed forms.

* Periodic box: total mass is conserved exactly (collision conserves rho,
  streaming permutes populations); total momentum too when lambda = mu, F = 0.
* Plane waves on a periodic box travel at the speeds fixed by the
  Lame-Navier equation (Eq. navier): c_d = sqrt((lambda + 2 mu)/rho),
  c_s = sqrt(mu/rho).  The lambda != mu case pins the source term of
  Eq. (sourceterm).
* 1-D impact of a bar (uniaxial strain) -- the textbook step-load solution:
  a traction step T on a free end sends a wave with sigma_xx = T,
  j_x = T/c_d, sigma_yy = lambda/(lambda + 2 mu) T; a clamped end reflects it
  with sigma_xx = 2T and j = 0; a wall moving at V sends j = rho0 V,
  sigma_xx = -rho0 c_d V; a shear traction sends sigma_xy = T, j_y = T/c_s.
  These pin Eqs. (bbcon), (abbcon) (and their curved forms, for any s/l)
  against exact values.
"""
import numpy as np
import pytest

MU = 1.0 / 3.0


def _periodic(oracle_mod, nx, ny, lam):
    nt, links = oracle_mod.geometry(nx, ny, edge_bc=(-1, -1, -1, -1))
    assert len(links) == 0
    return oracle_mod.Oracle(nt, links, [], lam=lam, mu=MU, periodic=(True, True))


@pytest.mark.parametrize("lam_over_mu", [1.0, 0.8])
def test_periodic_conservation(oracle_mod, lam_over_mu):
    rng = np.random.default_rng(1)
    o = _periodic(oracle_mod, 24, 16, lam_over_mu * MU)
    frest = oracle_mod.feq(1.0, (0, 0), (0, 0, 0))
    f0 = frest + rng.normal(0, 1e-4, (16, 24, 9))
    o.set_state(f0)
    C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
    m0 = f0.sum()
    p0 = np.einsum("yxi,ia->a", f0, C)
    o.step(60)
    f, _ = o.state()
    assert abs(f.sum() - m0) < 1e-11
    p1 = np.einsum("yxi,ia->a", f, C)
    if lam_over_mu == 1.0:
        np.testing.assert_allclose(p1, p0, atol=1e-12)
    else:
        # sum of (mu - lambda)/rho grad rho over the box is O(drho^2), not zero
        np.testing.assert_allclose(p1, p0, atol=1e-8)


def _wave_speed(oracle_mod, lam, kind, nx=256, steps=1100):
    o = _periodic(oracle_mod, nx, 1, lam)
    k = 2 * np.pi / nx
    x = np.arange(nx)
    f = np.zeros((1, nx, 9))
    for ix in range(nx):
        j = (1e-4 * np.sin(k * ix), 0.0) if kind == "P" else (0.0, 1e-4 * np.sin(k * ix))
        f[0, ix] = oracle_mod.feq(1.0, j, (0, 0, 0))
    o.set_state(f)
    comp = 0 if kind == "P" else 1
    a = []
    for _ in range(steps):
        F = o.fields()
        a.append((F["v"][comp, 0] * F["rho"][0] * np.sin(k * x)).sum())
        o.step(1)
    a = np.array(a)
    zc = [t + a[t] / (a[t] - a[t + 1]) for t in range(len(a) - 1) if a[t] * a[t + 1] < 0]
    period = 2 * np.diff(zc).mean()
    return nx / period


@pytest.mark.parametrize("lam_over_mu,kind", [(1.0, "P"), (1.0, "S"), (0.8, "P"),
                                              (1.0 / 0.3611 - 2.0, "P")])
def test_wave_speeds(oracle_mod, lam_over_mu, kind):
    lam = lam_over_mu * MU
    c = _wave_speed(oracle_mod, lam, kind)
    exact = np.sqrt(lam + 2 * MU) if kind == "P" else np.sqrt(MU)
    assert abs(c / exact - 1) < 1e-4, (c, exact)


def _bar(oracle_mod, lam, left, right, nx=256, steps=560, probe=128, q=None):
    nt, links = oracle_mod.geometry(nx, 1, edge_bc=(0, 1, -1, -1))
    if q is not None:
        sel = (links["node"] == nx - 1) & np.isin(links["dir"], [1, 5, 8])
        links["q"][sel] = q
        links["curved"][sel] = 1
    o = oracle_mod.Oracle(nt, links, [left, right], lam=lam, mu=MU, periodic=(False, True))
    j, s = [], []
    for _ in range(steps):
        F = o.fields()
        j.append(F["v"][:, 0, probe] * F["rho"][0, probe])
        s.append(F["sigma"][:, 0, probe])
        o.step(1)
    return np.array(j), np.array(s)


@pytest.mark.parametrize("lam_over_mu", [1.0, 0.8])
def test_bar_traction_step_and_clamped_reflection(oracle_mod, lam_over_mu):
    lam, T = lam_over_mu * MU, 1e-3
    cd = np.sqrt(lam + 2 * MU)
    D = dict(kind=oracle_mod.DIRICHLET, value=(0, 0))
    N = dict(kind=oracle_mod.NEUMANN, value=(T, 0))
    j, s = _bar(oracle_mod, lam, D, N, steps=620)
    t1 = slice(int(127.5 / cd) + 25, int(383.5 / cd) - 25)        # incident wave only
    t2 = slice(int(383.5 / cd) + 25, int(639.5 / cd) - 25)        # after the clamp
    tol = 1e-6 if lam_over_mu == 1.0 else 2e-3
    assert abs(j[t1, 0].mean() / (T / cd) - 1) < tol
    assert abs(s[t1, 0].mean() / T - 1) < tol
    assert abs(s[t1, 1].mean() / (lam / (lam + 2 * MU) * T) - 1) < tol
    assert abs(s[t1, 2]).max() < 1e-12
    assert abs(j[t2, 0].mean()) < tol * T / cd
    assert abs(s[t2, 0].mean() / (2 * T) - 1) < tol


def test_bar_moving_wall(oracle_mod):
    V = 1e-3
    D = dict(kind=oracle_mod.DIRICHLET, value=(V, 0))
    N = dict(kind=oracle_mod.NEUMANN, value=(0, 0))
    j, s = _bar(oracle_mod, MU, D, N, steps=360)
    w = slice(128 + 25, 384 - 25)
    assert abs(j[w, 0].mean() / V - 1) < 1e-6            # j = rho0 V
    assert abs(s[w, 0].mean() / (-V) - 1) < 1e-6         # sigma_xx = -rho0 c_d V


def test_bar_shear_traction(oracle_mod):
    T = 1e-3
    cs = np.sqrt(MU)
    F = dict(kind=oracle_mod.NEUMANN, value=(0, 0))
    N = dict(kind=oracle_mod.NEUMANN, value=(0, T))
    j, s = _bar(oracle_mod, MU, F, N, steps=560)
    w = slice(int(127.5 / cs) + 30, 560)
    assert abs(j[w, 1].mean() / (T / cs) - 1) < 1e-4
    assert abs(s[w, 2].mean() / T - 1) < 1e-4


@pytest.mark.parametrize("q", [0.1, 0.3, 0.7, 0.95])
@pytest.mark.parametrize("kind", ["neumann", "dirichlet"])
def test_curved_wall_plateau_is_exact_for_any_q(oracle_mod, q, kind):
    """Eqs. (bbnoncon), (abbnoncon): a wall at distance s = q l from the last
    node still imposes the exact boundary value behind the wave front."""
    T = 1e-3
    D = dict(kind=oracle_mod.DIRICHLET, value=(0, 0))
    right = (dict(kind=oracle_mod.NEUMANN, value=(T, 0)) if kind == "neumann"
             else dict(kind=oracle_mod.DIRICHLET, value=(-T, 0)))
    j, s = _bar(oracle_mod, MU, D, right, steps=360, q=q)
    w = slice(160, 340)
    if kind == "neumann":
        assert abs(j[w, 0].mean() / T - 1) < 1e-6
        assert abs(s[w, 0].mean() / T - 1) < 1e-6
    else:
        # the wall moves into the bar at speed T: j = -rho0 T, sigma_xx = -rho0 c_d T
        assert abs(j[w, 0].mean() / (-T) - 1) < 1e-6
        assert abs(s[w, 0].mean() / (-T) - 1) < 1e-6


def test_ramp_profile_follows_the_ramp(oracle_mod):
    """A traction ramped over t_ramp steps: during the ramp the end stress
    wave carries sigma_xx(t) = T min(t/t_ramp, 1) delayed by the travel time."""
    T, tr = 1e-3, 100.0
    D = dict(kind=oracle_mod.DIRICHLET, value=(0, 0))
    N = dict(kind=oracle_mod.NEUMANN, value=(T, 0), profile=oracle_mod.RAMP, t_ramp=tr)
    j, s = _bar(oracle_mod, MU, D, N, steps=340)
    # the probe sees the boundary history shifted by the travel time 127.5
    for t in (170, 200, 220):
        expected = T * min((t - 127.5) / tr, 1.0)
        assert abs(s[t, 0] - expected) < 0.03 * T, (t, s[t, 0], expected)
    assert abs(s[300:340, 0].mean() / T - 1) < 1e-3
