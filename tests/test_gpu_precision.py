"""GPU: the precision forms on the plate with a hole (Sec. 5.1 geometry).

The stress concentration at the rim of the hole is the quantity the plate
problem is about.  On the 256 x 128 downscale of the 1024 x 512 plate (hole
radius 16, Heaviside tension t* = 1e-3 on the left and right edges, wall-node
reading), the hoop stress sigma_tt = t.sigma.t (t the unit tangent of the
circle at the node's angle) is taken at every material node within 1.5
spacings of the rim, and its maximum over the rim divided by t* is compared
with the FP64 oracle's at t = 300 (the waves from both edges have met at the
hole and are reflecting) and t = 700 (the last step at which this downscale's
oracle run is still growth-free under the wall-node reading).

Bars: FP32 storage within 1e-5 of the oracle's concentration factor (the
parity bar), FP16 within 1e-3, BF16 within 1e-1 (measured 5.9e-2 at t = 700:
rounding to nearest in BF16's 8-bit significand keeps a population whose
change per step is below half its ulp where it is, and the run accumulates
those errors).
"""
import dataclasses

import numpy as np
import pytest

from paper_2208_04088_gb300 import workloads as W

pytestmark = pytest.mark.gpu
LOAD = 1e-3
TIMES = (300, 700)


def _rim_concentration(sigma, wl):
    cx, cy, r = wl.hole[0], wl.hole[1], wl.hole[2]
    y, x = np.mgrid[0:wl.ny, 0:wl.nx]
    d = np.hypot(x - cx, y - cy)
    rim = (d > r) & (d < r + 1.5)
    th = np.arctan2(y - cy, x - cx)
    t0, t1 = -np.sin(th), np.cos(th)
    sxx, syy, sxy = (np.asarray(s, np.float64) for s in sigma)
    stt = sxx * t0 * t0 + 2.0 * sxy * t0 * t1 + syy * t1 * t1
    return float(stt[rim].max()) / LOAD


@pytest.fixture(scope="module")
def plate():
    return dataclasses.replace(W.hole_plate(256, 128, 16.0, max(TIMES), load=LOAD),
                               wall_node=True)


@pytest.fixture(scope="module")
def oracle_scf(oracle_mod, plate):
    wl = plate
    nt, links = oracle_mod.geometry(**wl.geometry_args())
    o = oracle_mod.Oracle(nt, links, wl.bcs, lam=wl.lam, mu=wl.mu, tau=wl.tau,
                          wall_node=True)
    out = {}
    for t in TIMES:
        o.step(t - o.t)
        out[t] = _rim_concentration(o.fields()["sigma"], wl)
    o.close()
    return out


@pytest.mark.parametrize("storage,bar", [("f32", 1e-5), ("f16", 1e-3), ("bf16", 1e-1)])
def test_rim_stress_concentration(plate, oracle_scf, storage, bar):
    from paper_2208_04088_gb300 import _native as N
    s = N.Solver(N.desc_from_workload(plate, storage=storage))
    got = {}
    for t in TIMES:
        s.step(t - s.info()["time"])
        got[t] = _rim_concentration(s.fields_host()["sigma"], plate)
    s.close()
    # at t = 300 the two waves superpose at the hole and the dynamic
    # concentration overshoots the static Kirsch value 3 (oracle: 6.7)
    assert oracle_scf[300] > 3.0 and oracle_scf[700] > 1.0, oracle_scf
    for t in TIMES:
        assert abs(got[t] / oracle_scf[t] - 1.0) <= bar, (storage, t, got[t], oracle_scf[t])


def test_fp16_scale_follows_a_growing_run():
    """The 256 x 128 plate with a free hole grows in the FP64 oracle too (with
    the wall-node reading max |sigma| goes from 1.7e-3 at t = 500 to 1.2 at
    2000 and 53 at 2500: the curved traction-free rule is unstable there).  FP32
    storage keeps such a run finite; FP16 would overflow with the initial scale
    (65504 / 8192 leaves a factor 8000 above the load).  Its scale halves
    whenever a step stores a value above 8192, so after 3000 steps it has come
    down (measured: 4096 to 8), the populations stay finite (no non-finite
    moment is reported, as with FP32), and the stepping forms (two buffers, in
    place, batched) still agree bit for bit."""
    from paper_2208_04088_gb300 import _native as N
    wl = dataclasses.replace(W.hole_plate(256, 128, 16.0, 3000, load=LOAD), wall_node=True)
    s32 = N.Solver(N.desc_from_workload(wl))
    s32.step(wl.steps)
    s32.sync()
    s32.close()
    out = {}
    for in_place in (False, True):
        s = N.Solver(N.desc_from_workload(wl, storage="f16", in_place=in_place))
        scale0 = s.info()["storage_scale"]
        s.step(wl.steps)
        s.sync()                                # raises LBM_ERR_UNSTABLE if non-finite
        info = s.info()
        assert info["storage_scale"] <= scale0 / 64, (scale0, info["storage_scale"])
        out[in_place] = s.fields_host()
        s.close()
    b = N.Batch([N.desc_from_workload(wl, storage="f16"),
                 N.desc_from_workload(W.square_plate(64, 0), storage="f16")])
    b.step(wl.steps)
    b.sync()
    batched = b.fields_host(0)
    b.close()
    # the stored populations and their moments stay finite (the status words
    # are clear, and so is sigma, a moment); v = j/rho and its running sum u
    # may not, as the density of this diverged run crosses zero at some nodes
    # in FP32 too
    assert np.all(np.isfinite(out[False]["sigma"]))
    for k in ("u", "v", "sigma"):
        assert np.array_equal(out[False][k], out[True][k], equal_nan=True), k
        assert np.array_equal(out[False][k], batched[k], equal_nan=True), k
