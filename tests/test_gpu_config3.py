"""GPU: the 2048 x 2048 edge crack (Sec. 5.2) over its full 1500 steps against
the FP64 oracle on the full lattice.

The library runs the solve as bench.py times it (the default stepping form:
the temporally blocked kernel for FP32, one step per launch for 16-bit
storage).  The oracle runs the same 4.2 M-node lattice for 1500 steps, once per
wall reading (about 46 s on 16 host cores each), and its fields at t = 500 and
t = 1500 are shared by the tests of this module.

* FP32 storage: relative L2 <= 1e-5 on u, v and sigma over material nodes at
  t = 1500, with the wall-node reading that bench.py times.
* The paper's extrapolated wall values (Eqs. abbcon and abbnoncon with the
  extrapolated rho^bd) grow a density mode at the traction-free box edges that
  reaches max |sigma| of about 13 (13000 x the load) by t = 1500 in the oracle
  itself.  At t = 500 the library meets the 1e-5 bar.  At t = 1500 that run is
  so ill-conditioned that a relative change of 1e-7 in tau (the size of one
  FP32 rounding of an input) moves the oracle's u by 3 %, v by 2e-3 and sigma
  by 1.2e-5; no FP32 computation can be closer to it than that.  The bar there
  is therefore the oracle's own response to that change, field by field
  (measured library error: 8e-3, 8e-4, 9e-6).
* FP16 and BF16 storage: relative L2 against the oracle at t = 1500 within
  3e-3 (FP16) and 5e-2 (BF16; measured 2.0e-2 / 3.7e-2 / 3.3e-2 on u / v /
  sigma: rounding to nearest in an 8-bit significand keeps a population whose
  change per step is below half its ulp where it is, and those errors
  accumulate over the run), and the apparent stress intensity at t = 500 within
  1e-3 (FP16) and 1e-2 (BF16) of the oracle's.
"""
import dataclasses

import numpy as np
import pytest

from paper_2208_04088_gb300 import workloads as W

from helpers import compare

pytestmark = pytest.mark.gpu
T_K = 500


def _k_apparent(sigma_yy, length, y):
    sy = 0.5 * (np.asarray(sigma_yy[y], np.float64) + np.asarray(sigma_yy[y - 1], np.float64))
    xs = np.arange(length + 1, length + 11)
    return float((sy[xs] * np.sqrt(2 * np.pi * (xs - (length - 0.5)))).max())


def _workload(wall_node):
    return dataclasses.replace(W.CONFIG3, wall_node=wall_node)


def _oracle_run(oracle_mod, wl, tau=None):
    nt, links = oracle_mod.geometry(**wl.geometry_args())
    o = oracle_mod.Oracle(nt, links, wl.bcs, lam=wl.lam, mu=wl.mu, rho0=wl.rho0,
                          tau=wl.tau if tau is None else tau, wall_node=wl.wall_node)
    o.step(T_K)
    a = o.fields()
    o.step(wl.steps - T_K)
    b = o.fields()
    o.close()
    mask = nt.astype(bool)
    return ({"u": a["u"], "v": a["v"], "sigma": a["sigma"], "mask": mask},
            {"u": b["u"], "v": b["v"], "sigma": b["sigma"], "mask": mask})


@pytest.fixture(scope="module")
def oracle_wall_node(oracle_mod):
    return _oracle_run(oracle_mod, _workload(True))


def _gpu_run(wl, storage="f32"):
    from paper_2208_04088_gb300 import _native as N
    s = N.Solver(N.desc_from_workload(wl, storage=storage))
    info = s.info()
    s.step(T_K)
    a = s.fields_host()
    s.step(wl.steps - T_K)
    b = s.fields_host()
    s.sync()
    s.close()
    return a, b, info


def test_fp32_full_length_parity_wall_node(oracle_wall_node):
    from paper_2208_04088_gb300 import _native as N
    wl = _workload(True)
    a, b, info = _gpu_run(wl)
    assert info["time_block"] == N.LBM_TIME_BLOCK      # the benched stepping form
    ok, ol = oracle_wall_node
    err_k, err_l = compare(a, ok), compare(b, ol)
    assert all(e <= 1e-5 for e in err_k.values()), err_k
    assert all(e <= 1e-5 for e in err_l.values()), err_l
    for k in ("u", "v", "sigma"):
        assert np.all(b[k][..., ~ol["mask"]] == 0.0)
    length, y = wl.crack[0], wl.ny // 2
    ka, ko = _k_apparent(a["sigma"][1], length, y), _k_apparent(ok["sigma"][1], length, y)
    assert abs(ka / ko - 1.0) <= 1e-5, (ka, ko)


def test_fp32_full_length_parity_paper_rule(oracle_mod):
    wl = _workload(False)
    ok, ol = _oracle_run(oracle_mod, wl)
    a, b, _ = _gpu_run(wl)
    err_k = compare(a, ok)
    assert all(e <= 1e-5 for e in err_k.values()), err_k
    _, pert = _oracle_run(oracle_mod, wl, tau=wl.tau * (1.0 + 1e-7))
    sens = compare(pert, ol)
    err_l = compare(b, ol)
    assert all(err_l[k] <= max(1e-5, sens[k]) for k in err_l), (
        f"max|sigma| at t=1500 is {float(np.abs(ol['sigma']).max()):.3g}; oracle response "
        f"to a 1e-7 change of tau {sens}; library error {err_l}")


@pytest.mark.parametrize("storage,bound,k_bound", [("f16", 3e-3, 1e-3), ("bf16", 5e-2, 1e-2)])
def test_16bit_storage_full_length_accuracy(oracle_wall_node, storage, bound, k_bound):
    wl = _workload(True)
    a, b, info = _gpu_run(wl, storage)
    assert info["time_block"] == 1
    ok, ol = oracle_wall_node
    err = compare(b, ol)
    assert all(e <= bound for e in err.values()), err
    length, y = wl.crack[0], wl.ny // 2
    ka, ko = _k_apparent(a["sigma"][1], length, y), _k_apparent(ok["sigma"][1], length, y)
    assert abs(ka / ko - 1.0) <= k_bound, (ka, ko)
