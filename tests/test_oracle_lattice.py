"""Oracle pins: the single-node algebra of Sec. 3.

* Eq. (fieq): the equilibrium reproduces the prescribed moments rho, j, P
  (the defining property of the moment-chain equilibrium).
* Eq. (coll): collision conserves rho and P and shifts the momentum moment
  by S (so that j = sum f c + S/2 of Eq. (moments) is consistent).
* The rest populations against hand-derived fractions (tests/golden).
"""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]],
             dtype=np.float64)


def _moments(f):
    rho = f.sum()
    m = f @ C
    P = np.array([(f * C[:, 0] * C[:, 0]).sum(), (f * C[:, 1] * C[:, 1]).sum(),
                  (f * C[:, 0] * C[:, 1]).sum()])
    return rho, m, P


def test_rest_populations_match_golden(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "rest_populations.json")))
    fr = oracle_mod.feq(g["rho0"], (0, 0), (0, 0, 0))
    fractions = [float(eval(s)) for s in g["f_rest_fractions"]]
    np.testing.assert_allclose(fr, g["f_rest"], rtol=0, atol=1e-16)
    np.testing.assert_allclose(fr, fractions, rtol=0, atol=1e-16)


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_reproduces_moments(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    rho = 1.0 + rng.normal(0, 0.05)
    j = rng.normal(0, 0.05, 2)
    P = rng.normal(0, 0.05, 3)
    f = oracle_mod.feq(rho, j, P)
    r2, m2, P2 = _moments(f)
    assert abs(r2 - rho) < 1e-14
    np.testing.assert_allclose(m2, j, atol=1e-14)
    np.testing.assert_allclose(P2, P, atol=1e-14)


def test_equilibrium_is_linear_in_its_moments(oracle_mod):
    # Eq. (fieq) is affine in (rho, j, P): f(a + b) = f(a) + f(b) with the weights
    rng = np.random.default_rng(7)
    a = [rng.normal(), rng.normal(size=2), rng.normal(size=3)]
    b = [rng.normal(), rng.normal(size=2), rng.normal(size=3)]
    fa, fb = oracle_mod.feq(*a), oracle_mod.feq(*b)
    fab = oracle_mod.feq(a[0] + b[0], a[1] + b[1], a[2] + b[2])
    np.testing.assert_allclose(fab, fa + fb, atol=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_collision_invariants(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    frest = oracle_mod.feq(1.0, (0, 0), (0, 0, 0))
    f = frest + rng.normal(0, 1e-2, 9)
    S = rng.normal(0, 1e-2, 2)
    tau = 0.55
    fcol, j = oracle_mod.collide(f, S, tau)
    r0, m0, P0 = _moments(f)
    r1, m1, P1 = _moments(fcol)
    np.testing.assert_allclose(j, m0 + 0.5 * S, atol=1e-15)       # Eq. (moments)
    assert abs(r1 - r0) < 1e-14                                    # mass
    np.testing.assert_allclose(P1, P0, atol=1e-14)                 # Poisson stress
    np.testing.assert_allclose(m1, m0 + S, atol=1e-14)             # momentum gains S dt


def test_collision_at_equilibrium_without_source_is_identity(oracle_mod):
    f = oracle_mod.feq(1.01, (1e-3, -2e-3), (3e-3, -1e-3, 5e-4))
    fcol, _ = oracle_mod.collide(f, (0.0, 0.0), 0.55)
    np.testing.assert_allclose(fcol, f, atol=1e-15)
