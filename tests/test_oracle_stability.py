"""Oracle: long-run behaviour of the Neumann wall values.

The anti-bounce-back rules of Sec. 4 take the wall density (and, in this
reading, the wall stress for sigma_tt) by linear extrapolation along the link.
For a Poisson solid (lambda = mu) the density has no restoring force in the
bulk (the source of Eq. sourceterm vanishes), and the extrapolation feeds it
back at traction edges: the square plate develops a growing density mode after
about a thousand steps.  The paper's own runs stop before that (about 280 and
830 steps, Sec. 5).  Taking the wall values at the boundary node (the library's
LBM_WALL_NODE option) keeps straight edges bounded.  These tests pin both facts
so that a change to either rule shows up.
"""
import numpy as np
import pytest

from paper_2208_04088_gb300 import workloads as W


def _max_stress(oracle_mod, wl, steps, wall_node):
    nt, links = oracle_mod.geometry(**wl.geometry_args())
    o = oracle_mod.Oracle(nt, links, wl.bcs, lam=wl.lam, mu=wl.mu, tau=wl.tau,
                          wall_node=wall_node)
    out = []
    for _ in range(steps // 500):
        o.step(500)
        out.append(float(np.abs(o.fields()["sigma"]).max()))
    return out


def test_extrapolated_wall_values_grow_a_mode_on_the_square_plate(oracle_mod):
    s = _max_stress(oracle_mod, W.square_plate(64, 0), 2000, wall_node=False)
    assert s[-1] > 100 * s[0], s


def test_wall_node_values_keep_the_square_plate_bounded(oracle_mod):
    s = _max_stress(oracle_mod, W.square_plate(64, 0), 4000, wall_node=True)
    assert max(s) < 5e-3, s


@pytest.mark.parametrize("wall_node", [False, True])
def test_wall_node_option_keeps_exact_solutions(oracle_mod, wall_node):
    # 1-D traction step: behind the front the bar is uniform, so both readings agree
    nt, links = oracle_mod.geometry(256, 1, edge_bc=(0, 1, -1, -1))
    bcs = [dict(kind=0, value=(0, 0)), dict(kind=1, value=(1e-3, 0))]
    o = oracle_mod.Oracle(nt, links, bcs, lam=1 / 3, mu=1 / 3, periodic=(False, True),
                          wall_node=wall_node)
    acc = []
    for t in range(330):
        if 160 <= t < 330:
            F = o.fields()
            acc.append(F["sigma"][0, 0, 128])
        o.step(1)
    assert abs(np.mean(acc) / 1e-3 - 1) < 1e-6
