"""Oracle pin: the density-gradient source of Eq. (sourceterm) next to walls.

The source S = F + (mu - lambda)/rho grad rho needs grad rho at every material
node.  The paper gives no stencil; this library reads it as a central
difference along each axis, one-sided where exactly one axis neighbour is void,
outside the box or across a cut link, and zero where both are.  Every other
lambda != mu pin (plane waves, the 1-D impact plateaus, the uniform-stress
patch, rigid translation) has rho uniform at the nodes where the one-sided
forms apply, so a wrong sign or factor there would pass them.

tests/golden/source_gradient.json sets a non-uniform density on a 5 x 5 box
with a void node and cracks between material nodes, with f_i = w_i rho (zero
momentum).  One step then has a closed form (derived in the fixture): the
displacement is u(1) = S/(2 rho) at every node, and every pulled population is
f_i(x, 1) = w_i (rho(z) + 3 c_i.S(z)) with z = x - c_i, whatever tau is.  The
stencil of each node is written out in the fixture from the lattice layout, not
computed by the oracle.
"""
import json
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "source_gradient.json")
MU = 1.0 / 3.0
CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
W9 = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4


def _gold():
    with open(GOLD) as f:
        return json.load(f)


def _setup(oracle_mod, g):
    n = len(g["rho_milli"])
    (vx, vy), = g["void"]
    # a hole of radius 1/2 centred on the void node voids exactly that node
    nt, links = oracle_mod.geometry(n, n, edge_bc=(0, 0, 0, 0), hole=(float(vx), float(vy), 0.5, 0))
    expect_void = np.ones((n, n), dtype=np.uint8)
    expect_void[vy, vx] = 0
    assert np.array_equal(nt, expect_void)
    extra = np.zeros(len(g["cut_links"]), dtype=oracle_mod.LINK_DTYPE)
    for r, c in zip(extra, g["cut_links"]):
        r["node"] = c["y"] * n + c["x"]
        r["dir"] = c["dir"]
        r["bc"], r["bc2"] = 0, -1
        r["q"] = 0.5
        r["n0"], r["n1"] = c["n"]
    links = np.concatenate([links, extra])
    lam = g["lam_over_mu"] * MU
    o = oracle_mod.Oracle(nt, links, [dict(kind=oracle_mod.DIRICHLET, value=(0.0, 0.0))],
                          lam=lam, mu=MU, tau=g["tau"])
    rho = 1.0 + 1e-3 * np.array(g["rho_milli"], dtype=np.float64)
    rho[nt == 0] = 0.0
    f0 = rho[..., None] * np.array(W9)[None, None, :]
    o.set_state(f0)
    cut = {(int(l["node"]), int(l["dir"])) for l in links}
    return o, nt, rho, lam, cut


def _expected_source(g, rho, lam):
    """S at every material node from the stencils listed in the fixture."""
    S = {}
    for e in g["nodes"]:
        x, y = e["x"], e["y"]
        gr = []
        for ax, (dx, dy) in (("x", (1, 0)), ("y", (0, 1))):
            st = e["g" + ax]
            if st == "central":
                v = 0.5 * (rho[y + dy, x + dx] - rho[y - dy, x - dx])
            elif st == "forward":
                v = rho[y + dy, x + dx] - rho[y, x]
            elif st == "backward":
                v = rho[y, x] - rho[y - dy, x - dx]
            else:
                assert st == "zero"
                v = 0.0
            gr.append(v)
        S[(x, y)] = (MU - lam) / rho[y, x] * np.array(gr)
    return S


def test_fixture_covers_every_fallback():
    g = _gold()
    kinds = {(ax, e["g" + ax]) for e in g["nodes"] for ax in ("x", "y")}
    for ax in ("x", "y"):
        for st in ("central", "forward", "backward", "zero"):
            assert (ax, st) in kinds, (ax, st)
    whys = " ".join(e.get("gx_why", "") + e.get("gy_why", "") for e in g["nodes"])
    for cause in ("box edge", "void neighbour", "cut link between material nodes"):
        assert cause in whys


def test_displacement_after_one_step_is_half_the_source(oracle_mod):
    g = _gold()
    o, nt, rho, lam, _ = _setup(oracle_mod, g)
    S = _expected_source(g, rho, lam)
    o.step(1)
    _, u = o.state()
    o.close()
    assert len(S) == int(nt.sum())
    for (x, y), s in S.items():
        expect = s / (2.0 * rho[y, x])
        # |u| ~ 1e-6; the closed form holds to the rounding of the FP64 sums
        assert np.allclose(u[y, x], expect, rtol=1e-10, atol=1e-18), ((x, y), u[y, x], expect)
    # the one-sided and zero stencils are not the central one here: a central
    # difference with a missing neighbour taken as rho(x) would give half the
    # forward value, which the check above rejects
    assert abs(S[(2, 4)][0]) == 0.0 and abs(S[(4, 1)][1]) == 0.0
    assert abs(S[(3, 2)][0]) > 1e-4 and abs(S[(1, 4)][0]) > 1e-4


def test_pulled_populations_carry_the_upstream_source(oracle_mod):
    g = _gold()
    o, nt, rho, lam, cut = _setup(oracle_mod, g)
    S = _expected_source(g, rho, lam)
    n = nt.shape[0]
    o.step(1)
    f, _ = o.state()
    o.close()
    checked = 0
    for (x, y) in S:
        k = y * n + x
        # rest population: f_0(x, 1) = f_0^col(x) = w_0 rho(x)
        assert abs(f[y, x, 0] - W9[0] * rho[y, x]) < 1e-15
        for i in range(1, 9):
            if (k, OPP[i]) in cut:
                continue  # given by a boundary rule, not pulled
            zx, zy = x - CX[i], y - CY[i]
            sz = S[(zx, zy)]
            expect = W9[i] * (rho[zy, zx] + 3.0 * (CX[i] * sz[0] + CY[i] * sz[1]))
            assert abs(f[y, x, i] - expect) < 1e-15, ((x, y), i, f[y, x, i], expect)
            checked += 1
    assert checked > 100
