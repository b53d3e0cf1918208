"""Oracle pins: the boundary rules of Sec. 4 against exact solutions.

* Zero load: the rest state stays at rest under every rule.
* Rigid translation: f = f^eq(rho0, rho0 v, 0) with j* = rho0 v on every wall
  is an exact solution of Eqs. (bbcon)/(bbnoncon) for any wall distance.
* Patch test: a uniform stress sigma0 with t* = sigma0 n on every wall is an
  exact solution of Eqs. (abbcon)/(abbnoncon) -- this pins the rotation of
  Eq. (trafocauchy), the Poisson stress of Eq. (bcchainneum) and the
  extrapolated sigma_tt for any wall normal and distance, for lambda != mu too.
* Both exact states on a seeded fragmented solid (isolated nodes, cracks
  between material nodes, random q and normals, missing upstream nodes).
* Curved forms with s = l/2 reduce bit-exactly to the lattice-conforming ones.
* Linearity and mirror symmetry of the hole plate.
* Hand-derived first-step populations (tests/golden/first_step.json).
"""
import json
import os

import numpy as np
import pytest

from paper_2208_04088_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
MU = 1.0 / 3.0


def _run(oracle_mod, wl, steps, bcs=None, links_edit=None, lam=None):
    nt, links = oracle_mod.geometry(**wl.geometry_args())
    if links_edit is not None:
        links = links_edit(links)
    o = oracle_mod.Oracle(nt, links, bcs if bcs is not None else wl.bcs,
                          lam=wl.lam if lam is None else lam, mu=wl.mu, tau=wl.tau)
    o.step(steps)
    return o, nt, links


def test_rest_state_stays_at_rest(oracle_mod):
    wl = W.hole_plate(64, 48, 9.0, 0)
    bcs = [dict(kind=0, value=(0, 0)), dict(kind=1, value=(0, 0))]
    o, nt, _ = _run(oracle_mod, wl, 200, bcs=bcs)
    F = o.fields()
    # only rounding noise of the absolute-f arithmetic (f ~ 1) may appear
    assert np.abs(F["u"]).max() < 2e-12
    assert np.abs(F["v"]).max() < 2e-13
    assert np.abs(F["sigma"]).max() < 2e-13


@pytest.mark.parametrize("lam_over_mu", [1.0, 0.8])
def test_rigid_translation_is_exact(oracle_mod, lam_over_mu):
    v = np.array([3e-4, -2e-4])
    wl = W.hole_plate(48, 40, 7.3, 0, lam_over_mu=lam_over_mu)
    nt, links = oracle_mod.geometry(**wl.geometry_args())
    bcs = [dict(kind=oracle_mod.DIRICHLET, value=tuple(v))] * 2
    o = oracle_mod.Oracle(nt, links, bcs, lam=wl.lam, mu=MU)
    f0 = np.zeros((wl.ny, wl.nx, 9))
    f0[nt.astype(bool)] = oracle_mod.feq(1.0, v, (0, 0, 0))
    o.set_state(f0)
    n = 60
    o.step(n)
    F = o.fields()
    m = nt.astype(bool)
    assert (links["curved"] == 1).sum() > 20
    for a in range(2):
        np.testing.assert_allclose(F["v"][a][m], v[a], rtol=0, atol=3e-14)
        np.testing.assert_allclose(F["u"][a][m], n * v[a], rtol=1e-10, atol=0)
    assert np.abs(F["sigma"][:, m]).max() < 3e-14


@pytest.mark.parametrize("lam_over_mu", [1.0, 0.8])
def test_patch_uniform_stress_is_exact(oracle_mod, lam_over_mu):
    sig0 = np.array([[1.0e-3, 4.0e-4], [4.0e-4, -6.0e-4]])
    wl = W.hole_plate(48, 40, 7.3, 0, lam_over_mu=lam_over_mu)
    lam = wl.lam
    nt, links = oracle_mod.geometry(**wl.geometry_args())
    # every wall carries t* = sigma0 n (a stress boundary condition)
    bcs = [dict(kind=oracle_mod.STRESS, value=(sig0[0, 0], sig0[1, 1], sig0[0, 1]))] * 2
    o = oracle_mod.Oracle(nt, links, bcs, lam=lam, mu=MU)
    # plane strain: tr(sigma) = 2 (lambda + mu) div u; rho = rho0 (1 - div u)
    divu = np.trace(sig0) / (2 * (lam + MU))
    rho = 1.0 - divu
    P = -sig0 + (lam - MU) * divu * np.eye(2)
    f0 = np.zeros((wl.ny, wl.nx, 9))
    f0[nt.astype(bool)] = oracle_mod.feq(rho, (0, 0), (P[0, 0], P[1, 1], P[0, 1]))
    o.set_state(f0)
    o.step(60)
    F = o.fields()
    m = nt.astype(bool)
    np.testing.assert_allclose(F["sigma"][0][m], sig0[0, 0], atol=3e-14)
    np.testing.assert_allclose(F["sigma"][1][m], sig0[1, 1], atol=3e-14)
    np.testing.assert_allclose(F["sigma"][2][m], sig0[0, 1], atol=3e-14)
    assert np.abs(F["v"][:, m]).max() < 3e-14


FRAGMENTED = [(150, 45, 7, 0.2, 0.05), (40, 30, 3, 0.6, 0.05), (33, 17, 1, 0.0, 0.3)]


def _fragmented_links(oracle_mod, cols):
    links = np.zeros(len(cols["node"]), dtype=oracle_mod.LINK_DTYPE)
    for k in ("node", "dir", "bc", "bc2", "q", "n0", "n1"):
        links[k] = cols[k]
    links["curved"] = 1
    return links


@pytest.mark.parametrize("lam_over_mu", [1.0, 0.8])
@pytest.mark.parametrize("args", FRAGMENTED, ids=["wide", "sparse", "cracked"])
def test_exact_states_on_a_fragmented_solid(oracle_mod, args, lam_over_mu):
    """Rigid translation and the uniform-stress patch on the seeded fragmented
    solid.  The solid has isolated nodes with eight cut links, cracks between
    material nodes, wall distances anywhere in (0, 1], random unit normals and
    missing upstream nodes.  Both states are exact for any wall distance and
    any normal: t* = sigma0 n rotated to the wall frame, with sigma_tt taken
    from the material, gives back sigma0.  The patch is checked after 10 steps.
    With free single nodes the Neumann rules are unstable, so rounding noise in
    it grows about a millionfold per 20 steps."""
    nx, ny, seed, vf, cf = args
    nt, cols = W.fragmented_solid(nx, ny, seed, void_frac=vf, crack_frac=cf, nbcs=2)
    links = _fragmented_links(oracle_mod, cols)
    m = nt.astype(bool)
    lam = lam_over_mu * MU
    v = np.array([3e-4, -2e-4])
    o = oracle_mod.Oracle(nt, links, [dict(kind=oracle_mod.DIRICHLET, value=tuple(v))] * 2,
                          lam=lam, mu=MU)
    f0 = np.zeros(nt.shape + (9,))
    f0[m] = oracle_mod.feq(1.0, v, (0, 0, 0))
    o.set_state(f0)
    o.step(60)
    F = o.fields()
    for a in range(2):
        np.testing.assert_allclose(F["v"][a][m], v[a], rtol=0, atol=5e-14)
        np.testing.assert_allclose(F["u"][a][m], 60 * v[a], rtol=1e-10, atol=0)
    assert np.abs(F["sigma"][:, m]).max() < 5e-14

    sig0 = np.array([[1.0e-3, 4.0e-4], [4.0e-4, -6.0e-4]])
    bcs = [dict(kind=oracle_mod.STRESS, value=(sig0[0, 0], sig0[1, 1], sig0[0, 1]))] * 2
    o = oracle_mod.Oracle(nt, links, bcs, lam=lam, mu=MU)
    divu = np.trace(sig0) / (2 * (lam + MU))
    P = -sig0 + (lam - MU) * divu * np.eye(2)
    f0 = np.zeros(nt.shape + (9,))
    f0[m] = oracle_mod.feq(1.0 - divu, (0, 0), (P[0, 0], P[1, 1], P[0, 1]))
    o.set_state(f0)
    o.step(10)
    F = o.fields()
    for c, ref in enumerate((sig0[0, 0], sig0[1, 1], sig0[0, 1])):
        np.testing.assert_allclose(F["sigma"][c][m], ref, rtol=0, atol=2e-13)
    assert np.abs(F["v"][:, m]).max() < 2e-13


def test_curved_rules_at_half_link_equal_conforming_bitwise(oracle_mod):
    wl = W.square_plate(40, 0)
    bcs = [dict(kind=0, value=(2e-4, -1e-4)), dict(kind=1, value=(1e-3, 3e-4)),
           dict(kind=1, value=(-2e-4, 1e-4))]

    def as_curved(links):
        links = links.copy()
        links["curved"] = 1
        assert np.all(links["q"] == 0.5)
        return links

    a, _, _ = _run(oracle_mod, wl, 150, bcs=bcs)
    b, _, _ = _run(oracle_mod, wl, 150, bcs=bcs, links_edit=as_curved)
    fa, ua = a.state()
    fb, ub = b.state()
    assert np.array_equal(fa, fb) and np.array_equal(ua, ub)


def test_linearity_and_superposition(oracle_mod):
    # lambda = mu: the scheme is affine in f and linear in the boundary data, so
    # the moments j = rho v, rho - rho0 and sigma are linear in the load
    # (v = j/rho and u = sum j/rho are not: they divide by the density)
    wl = W.hole_plate(48, 32, 6.0, 0)
    nt, links = oracle_mod.geometry(**wl.geometry_args())

    def run(pl, sh):
        bcs = [dict(kind=oracle_mod.PRESSURE, value=(pl,)), dict(kind=oracle_mod.NEUMANN, value=(0, sh))]
        o = oracle_mod.Oracle(nt, links, bcs, lam=MU, mu=MU)
        o.step(120)
        return o.fields()

    def lin(F):
        return {"j": F["v"] * F["rho"], "drho": F["rho"] - 1.0 * (nt > 0), "sigma": F["sigma"]}

    A, B, AB, A2 = (lin(run(-1e-3, 0)), lin(run(0, 4e-4)), lin(run(-1e-3, 4e-4)),
                    lin(run(-2e-3, 0)))
    for key in ("j", "drho", "sigma"):
        scale = np.abs(AB[key]).max()
        assert np.abs(A2[key] - 2 * A[key]).max() < 1e-10 * scale
        assert np.abs(AB[key] - A[key] - B[key]).max() < 1e-10 * scale


def test_hole_plate_mirror_symmetry(oracle_mod):
    wl = W.hole_plate(60, 44, 8.0, 300)
    o, nt, _ = _run(oracle_mod, wl, wl.steps)
    F = o.fields()
    ux, uy = F["u"]
    sxx, syy, sxy = F["sigma"]
    s = np.abs(F["u"]).max()
    # x-mirror: u_x odd, u_y even; y-mirror: u_x even, u_y odd
    assert np.abs(ux + ux[:, ::-1]).max() < 1e-10 * s
    assert np.abs(uy - uy[:, ::-1]).max() < 1e-10 * s
    assert np.abs(ux - ux[::-1, :]).max() < 1e-10 * s
    assert np.abs(uy + uy[::-1, :]).max() < 1e-10 * s
    ss = np.abs(F["sigma"]).max()
    assert np.abs(sxx - sxx[::-1, ::-1]).max() < 1e-10 * ss
    assert np.abs(sxy + sxy[:, ::-1]).max() < 1e-10 * ss


def _first_step(oracle_mod, edge, value, kind, q=None):
    nx, ny = 12, 8
    # edge under test gets bc 1, the others are clamped (bc 0); the probe node
    # sits mid-edge so its neighbours are away from other walls
    eb = [0, 0, 0, 0]
    eb[{"left": 0, "right": 1}[edge]] = 1
    nt, links = oracle_mod.geometry(nx, ny, edge_bc=tuple(eb))
    if q is not None:
        sel = links["bc"] == 1
        links["q"][sel] = q
        links["curved"][sel] = 1
    bcs = [dict(kind=0, value=(0, 0)), dict(kind=kind, value=value)]
    o = oracle_mod.Oracle(nt, links, bcs, lam=MU, mu=MU)
    o.step(1)
    f, _ = o.state()
    frest = oracle_mod.feq(1.0, (0, 0), (0, 0, 0))
    x = nx - 1 if edge == "right" else 0
    return f[ny // 2, x] - frest, o.fields(), (ny // 2, x)


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLD, "first_step.json")))["cases"],
                         ids=lambda c: c["name"])
def test_first_step_golden(oracle_mod, case):
    if "traction" in case:
        df, F, (y, x) = _first_step(oracle_mod, case["edge"], case["traction"], oracle_mod.NEUMANN)
    else:
        df, F, (y, x) = _first_step(oracle_mod, case["edge"], case["wall_velocity"],
                                    oracle_mod.DIRICHLET, q=case.get("q"))
    expected = np.zeros(9)
    for k, v in case["delta_f_values"].items():
        expected[int(k)] = v
    np.testing.assert_allclose(df, expected, rtol=0, atol=1e-15)
    fx = case.get("fields_at_node_after_one_step", {})
    if "sigma_xx" in fx:
        assert abs(F["sigma"][0, y, x] - fx["sigma_xx"]) < 1e-15
        assert abs(F["sigma"][1, y, x] - fx["sigma_yy"]) < 1e-15
        assert abs(F["sigma"][2, y, x] - fx["sigma_xy"]) < 1e-15
    if "rho" in fx:
        assert abs(F["rho"][y, x] - fx["rho"]) < 1e-15
        assert abs(F["v"][0, y, x] * F["rho"][y, x] - fx["j_x"]) < 1e-15


def test_corner_link_first_step_golden(oracle_mod):
    case = json.load(open(os.path.join(GOLD, "first_step.json")))["corner_case"]
    nx, ny = 10, 8
    nt, links = oracle_mod.geometry(nx, ny, edge_bc=(0, 1, 0, 2))
    bcs = [dict(kind=0, value=(0, 0)), dict(kind=1, value=case["right_traction"]),
           dict(kind=1, value=case["top_traction"])]
    o = oracle_mod.Oracle(nt, links, bcs, lam=MU, mu=MU)
    o.step(1)
    f, _ = o.state()
    frest = oracle_mod.feq(1.0, (0, 0), (0, 0, 0))
    df = f[ny - 1, nx - 1] - frest
    assert abs(df[7] - case["delta_f7_value"]) < 1e-15
