"""GPU checks at the full sizes of the benchmark configurations, in the launch
configuration bench.py times (replayed graphs, boundary kernel beside the
interior kernel).

* 2048^2 edge crack: at t = 300 the disturbance has travelled at most 300 nodes
  (one node per step), so the FP64 oracle on a crop that reaches more than 300
  nodes beyond the crack computes the same fields as on the full lattice; the
  GPU run of the full lattice must match it there and be exactly zero outside
  the light cone.  At t = 500 (< l_c/c_d = 512) the stress intensity ahead of
  the tip is compared with Freund's K_I^0 (Sec. 5.2).
* 1024 x 512 plate with hole: full-field parity with the oracle at t = 600.
"""
import numpy as np
import pytest

from paper_2208_04088_gb300 import workloads as W

from helpers import compare, rel_l2

pytestmark = pytest.mark.gpu


def _gpu_solver(wl, storage="f32"):
    from paper_2208_04088_gb300 import _native as N
    return N.Solver(N.desc_from_workload(wl, storage=storage))


def test_config3_crack_fullsize_against_cropped_oracle(oracle_mod):
    wl = W.CONFIG3
    t = 300
    s = _gpu_solver(wl)
    s.step(t)
    G = s.fields_host()
    # the crop: columns [0, 512 + 320), rows [1024 - 320, 1024 + 320)
    y0, y1, x1 = 1024 - 320, 1024 + 320, 512 + 320
    crop = W.edge_crack(x1, 512, t, ny=y1 - y0)
    nt, links = oracle_mod.geometry(**crop.geometry_args())
    # inner crop edges are not walls of the full problem: nothing reaches them
    # by t = 300, and the crop keeps the left edge and the crack as they are
    o = oracle_mod.Oracle(nt, links, crop.bcs, lam=crop.lam, mu=crop.mu, tau=crop.tau)
    o.step(t)
    F = o.fields()
    mask = np.ones((y1 - y0, x1), dtype=bool)
    sub = {k: G[k][:, y0:y1, :x1] for k in ("u", "v", "sigma")}
    err = {k: rel_l2(sub[k], F[k], mask) for k in ("u", "v", "sigma")}
    assert all(e <= 1e-5 for e in err.values()), err
    # outside the light cone of the loaded crack faces everything is still zero
    for k in ("u", "v", "sigma"):
        assert np.all(G[k][:, :, 512 + 302:] == 0.0)
        assert np.all(G[k][:, : 1024 - 302, :] == 0.0)
        assert np.all(G[k][:, 1024 + 302:, :] == 0.0)
    s.close()


def test_config3_crack_fullsize_stress_intensity_and_symmetry(oracle_mod):
    wl = W.CONFIG3
    s = _gpu_solver(wl)
    Lc, y = 512, 1024
    s.step(500)
    G = s.fields_host()
    sy = 0.5 * (G["sigma"][1, y] + G["sigma"][1, y - 1]).astype(np.float64)
    xs = np.arange(Lc + 1, Lc + 11)
    k_app = sy[xs] * np.sqrt(2 * np.pi * (xs - (Lc - 0.5)))
    ratio = k_app.max() / oracle_mod.freund_ki0(500, 1e-3, wl.nu, wl.cd)
    assert 0.93 < ratio < 1.03, ratio
    # mirror symmetry about the crack plane y = 1023.5
    ux, uy = G["u"].astype(np.float64)
    scale = np.abs(G["u"]).max()
    assert np.abs(ux - ux[::-1, :]).max() < 1e-4 * scale
    assert np.abs(uy + uy[::-1, :]).max() < 1e-4 * scale
    # the full run stays finite
    s.step(wl.steps - 500)
    s.sync()
    s.close()


def test_config2_hole_plate_fullsize_parity(oracle_mod):
    wl = W.CONFIG2
    t = 600
    s = _gpu_solver(wl)
    s.step(t)
    G = s.fields_host()
    s.close()
    nt, links = oracle_mod.geometry(**wl.geometry_args())
    o = oracle_mod.Oracle(nt, links, wl.bcs, lam=wl.lam, mu=wl.mu, tau=wl.tau)
    o.step(t)
    F = o.fields()
    F["mask"] = nt.astype(bool)
    err = compare(G, F)
    assert all(e <= 1e-5 for e in err.values()), err
