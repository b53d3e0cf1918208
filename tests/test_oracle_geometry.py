"""Oracle pins: geometry classification (Sec. 4, Fig. boundnoncon; the wall
distance s_i of Eqs. (bbnoncon), (abbnoncon)) checked by brute force.

Nodes sit at integer (x, y); the box is [-1/2, nx - 1/2] x [-1/2, ny - 1/2],
so box edges cut links at mid-link (s/l = 1/2).  A hole link is cut iff its
end node is void; s/l is where the link first meets the circle.
"""
import numpy as np
import pytest

C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])


def test_box_link_count_and_corners(oracle_mod):
    for nx, ny in [(64, 64), (17, 9), (3, 2)]:
        nt, links = oracle_mod.geometry(nx, ny, edge_bc=(0, 1, 2, 3))
        assert nt.all()
        # brute force: every (node, direction) whose target leaves the box
        expect = sum(1 for y in range(ny) for x in range(nx) for i in range(1, 9)
                     if not (0 <= x + C[i, 0] < nx and 0 <= y + C[i, 1] < ny))
        assert len(links) == expect
        assert np.all(links["q"] == 0.5) and np.all(links["curved"] == 0)
        corner = links["bc2"] >= 0
        assert corner.sum() == 4
        # corner links are the outward diagonals of the corner nodes
        for L in links[corner]:
            x, y = L["node"] % nx, L["node"] // nx
            assert x in (0, nx - 1) and y in (0, ny - 1)
            assert L["n0"] == C[L["dir"], 0] and L["n1"] == C[L["dir"], 1]
            assert L["bc"] == (0 if x == 0 else 1) and L["bc2"] == (2 if y == 0 else 3)
        # ordering: node row-major, then direction
        key = links["node"].astype(np.int64) * 9 + links["dir"]
        assert np.all(np.diff(key) > 0)


@pytest.mark.parametrize("nx,ny,R", [(64, 48, 9.0), (256, 128, 16.0), (101, 77, 12.5)])
def test_hole_classification_brute_force(oracle_mod, nx, ny, R):
    cx, cy = 0.5 * (nx - 1), 0.5 * (ny - 1)
    nt, links = oracle_mod.geometry(nx, ny, edge_bc=(0, 0, 1, 1), hole=(cx, cy, R, 2))
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    inside = (X - cx) ** 2 + (Y - cy) ** 2 < R * R
    assert np.array_equal(nt == 0, inside)
    hole = links[links["bc"] == 2]
    # every (material node, direction) pointing at a void node, and nothing else
    expect = set()
    for y in range(ny):
        for x in range(nx):
            if inside[y, x]:
                continue
            for i in range(1, 9):
                tx, ty = x + C[i, 0], y + C[i, 1]
                if 0 <= tx < nx and 0 <= ty < ny and inside[ty, tx]:
                    expect.add((y * nx + x, i))
    assert set(zip(hole["node"].tolist(), hole["dir"].tolist())) == expect
    assert np.all(hole["curved"] == 1)
    for L in hole:
        x, y = L["node"] % nx, L["node"] // nx
        c = C[L["dir"]]
        q = L["q"]
        assert 0.0 < q <= 1.0
        w = np.array([x, y]) + q * c
        assert abs(np.hypot(w[0] - cx, w[1] - cy) - R) < 1e-12 * R
        # first crossing: the link stays outside the circle before q
        s = np.linspace(0.0, q, 50)[:-1]
        assert np.all(np.hypot(x + s * c[0] - cx, y + s * c[1] - cy) > R)
        n = np.array([L["n0"], L["n1"]])
        assert abs(np.hypot(*n) - 1.0) < 1e-12
        # outward normal of the material points to the centre
        np.testing.assert_allclose(n, (np.array([cx, cy]) - w) / R, atol=1e-14)


def test_edge_crack_links(oracle_mod):
    nx, ny, Lc = 40, 20, 11
    nt, links = oracle_mod.geometry(nx, ny, edge_bc=(0, 0, 0, 0), crack=(Lc, 1))
    crack = links[(links["bc"] == 1) | (links["bc2"] == 1)]
    ys = 0.5 * ny - 0.5
    expect = set()
    for y in (ny // 2 - 1, ny // 2):
        for x in range(nx):
            for i in range(1, 9):
                if C[i, 1] == 0:
                    continue
                ymid = y + 0.5 * C[i, 1]
                xmid = x + 0.5 * C[i, 0]
                if ymid == ys and xmid < Lc - 0.5:
                    expect.add((y * nx + x, i))
    assert set(zip(crack["node"].tolist(), crack["dir"].tolist())) == expect
    for L in crack:
        y = L["node"] // nx
        assert L["n1"] == (1.0 if y == ny // 2 - 1 else -1.0)
        assert L["q"] == 0.5
    # the two links through the crack mouth are corners of the left edge and the crack
    mouth = crack[crack["bc2"] == 1]
    assert len(mouth) == 2 and np.all(mouth["bc"] == 0) and np.all(mouth["n0"] == -1.0)
    # links crossing exactly at the tip (x = Lc - 1/2) are not cut
    tipnode = (ny // 2 - 1) * nx + (Lc - 1)
    assert not np.any((crack["node"] == tipnode) & (crack["dir"] == 5))


def test_rejects_bad_arguments(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.geometry(10, 9, crack=(3, 0))      # odd ny has no mid-row plane
    with pytest.raises(ValueError):
        oracle_mod.geometry(10, 10, edge_bc=(-1, 0, 0, 0))   # half-periodic axis


def test_centre_crack_links(oracle_mod):
    nx, ny, Lc, x0 = 40, 20, 11, 14
    nt, links = oracle_mod.geometry(nx, ny, edge_bc=(0, 0, 0, 0), crack=(Lc, 1, x0))
    crack = links[(links["bc"] == 1) | (links["bc2"] == 1)]
    ys = 0.5 * ny - 0.5
    expect = set()
    for y in (ny // 2 - 1, ny // 2):
        for x in range(nx):
            for i in range(1, 9):
                if C[i, 1] == 0:
                    continue
                xm = x + 0.5 * C[i, 0]
                if y + 0.5 * C[i, 1] == ys and x0 - 0.5 < xm < x0 + Lc - 0.5:
                    expect.add((y * nx + x, i))
    assert set(zip(crack["node"].tolist(), crack["dir"].tolist())) == expect
    assert np.all(crack["bc2"] == -1)   # no corner: the crack is away from the edges
    # both tips: diagonal links crossing exactly at x0 - 1/2 and x0 + Lc - 1/2 stay uncut
    below = (ny // 2 - 1) * nx
    assert not np.any((crack["node"] == below + x0 - 1) & (crack["dir"] == 5))
    assert not np.any((crack["node"] == below + x0 + Lc - 1) & (crack["dir"] == 5))
