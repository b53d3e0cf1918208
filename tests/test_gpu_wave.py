"""GPU: temporally blocked stepping (lbm_desc.time_block = LBM_TIME_BLOCK).

The blocked kernel carries LBM_TIME_BLOCK steps of a strip of the lattice in
shared memory per launch.  Per node and level it performs the one-step
arithmetic (interior: the same collision; boundary nodes: the cooperative
boundary update with its sums in the same order), so its fields must be
bit-identical to time_block = 1 after any number of steps -- single launches,
replayed graphs and the one-step remainder alike.  It is also compared with
the FP64 oracle at the FP32 tolerance.
"""
import dataclasses

import numpy as np
import pytest

from paper_2208_04088_gb300 import _native as N
from paper_2208_04088_gb300 import workloads as W

from helpers import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
TB = N.LBM_TIME_BLOCK


def _with(wl, **kw):
    return dataclasses.replace(wl, **kw)


def _moving_wall_plate():
    # Dirichlet edge with a ramped wall velocity (the boundary time of every level matters)
    wl = W.square_plate(160, 0)
    wl.bcs = [W.bc(W.DIRICHLET, (2e-4, -1e-4), W.RAMP, 13.0), W.bc(W.TRACTION, (1e-3, 5e-4)),
              W.bc(W.TRACTION, (0.0, 0.0))]
    return wl


CASES = [
    _with(W.hole_plate(256, 128, 16.0, 0), name="hole_256x128_extrapolate"),
    _with(W.hole_plate(256, 128, 16.0, 0), wall_node=True, name="hole_256x128_node"),
    _with(W.hole_plate(300, 140, 23.5, 0, profile=W.RAMP, t_ramp=17.0), name="hole_ramp_300x140"),
    _with(W.square_plate(128, 0), name="square_128"),
    _moving_wall_plate(),
    _with(W.edge_crack(256, 64, 0), name="edge_crack_256_L64"),
    _with(W.edge_crack(256, 64, 0), wall_node=True, name="edge_crack_256_L64_node"),
    _with(W.centre_crack(32, 0), name="centre_crack_128_L32"),
]


@pytest.mark.parametrize("steps", [8, 45, 77])
@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_blocked_bit_identical_to_one_step(wl, steps):
    a = run_gpu(wl, steps, time_block=1)
    b = run_gpu(wl, steps, time_block=TB)
    assert a["info"]["time_block"] == 1 and b["info"]["time_block"] == TB
    for k in ("u", "v", "sigma"):
        assert np.array_equal(a[k], b[k]), (k, float(np.abs(a[k] - b[k]).max()))


def test_blocked_bit_identical_in_chunks():
    # a run split across calls (partial blocks, graph chunks, remainders) ends
    # in the same state as one call
    wl = CASES[0]
    a = run_gpu(wl, 100, time_block=1)
    b = run_gpu(wl, 100, time_block=TB, chunks=[3, 40, 9, 48])
    for k in ("u", "v", "sigma"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("wl,steps", [(_with(W.square_plate(128, 0), wall_node=True), 500),
                                      (W.hole_plate(256, 128, 16.0, 0), 500),
                                      (_with(W.edge_crack(256, 64, 0), wall_node=True), 300)],
                         ids=["square_128_node", "hole_256x128", "edge_crack_256_node"])
def test_blocked_parity_with_oracle(oracle_mod, wl, steps):
    gpu = run_gpu(wl, steps, time_block=TB)
    assert gpu["info"]["time_block"] == TB
    err = compare(gpu, run_oracle(oracle_mod, wl, steps))
    assert all(e <= 1e-5 for e in err.values()), err


def test_blocked_full_size_crack_bit_identical():
    # the 2048^2 edge crack (L = 512) over its 1500 steps, as the benchmark runs it
    wl = _with(W.CONFIG3, wall_node=True)
    a = run_gpu(wl, wl.steps, time_block=1)
    b = run_gpu(wl, wl.steps, time_block=TB)
    for k in ("u", "v", "sigma"):
        assert np.array_equal(a[k], b[k]), k


def test_blocked_timing_mode_and_launch_count():
    wl = CASES[0]
    d = N.desc_from_workload(wl, time_block=TB)
    s = N.Solver(d)
    before = s.info()["kernel_launches"]
    s.step(64)  # two replayed graphs of 32 steps: 4 blocked launches + 1 advance each
    assert s.info()["kernel_launches"] - before == 2 * (32 // TB + 1)
    s.set_timing(True)
    s.step(2 * TB + 3)
    t = s.timing()
    s.close()
    assert t["steps"] == 2 * TB + 3
    assert t["interior_ms"] > 0.0


def test_blocked_reports_non_finite():
    wl = W.square_plate(128, 0, load=3e38)  # the moment sums overflow FP32
    for tb in (1, TB):
        d = N.desc_from_workload(wl, time_block=tb)
        s = N.Solver(d)
        s.step(40)
        with pytest.raises(N.LbmError, match="LBM_ERR_UNSTABLE"):
            s.sync()
        s.close()


# lambda != mu: the source needs grad rho; the blocked kernel carries 4 steps
# per launch (densities of each level formed two rows ahead)
PAPER = W.CRACK_PAPER_LAM_OVER_MU


def _moving_wall_plate_nonpoisson():
    wl = _moving_wall_plate()
    wl.lam_over_mu = W.PLATE_NONPOISSON_LAM_OVER_MU
    wl.name = "moving_wall_160_nonpoisson"
    return wl


GRAD_CASES = [
    _with(W.hole_plate(256, 128, 16.0, 0, lam_over_mu=0.8), name="hole_256x128_nonpoisson"),
    _with(W.hole_plate(256, 128, 16.0, 0, lam_over_mu=0.8), wall_node=True,
          name="hole_256x128_nonpoisson_node"),
    _with(W.edge_crack(256, 64, 0, lam_over_mu=PAPER), name="edge_crack_256_L64_paper"),
    _with(W.centre_crack(32, 0, lam_over_mu=PAPER), name="centre_crack_128_L32_paper"),
    _moving_wall_plate_nonpoisson(),
]


@pytest.mark.parametrize("steps", [4, 37, 77])
@pytest.mark.parametrize("wl", GRAD_CASES, ids=lambda w: w.name)
def test_blocked_nonpoisson_bit_identical_to_one_step(wl, steps):
    a = run_gpu(wl, steps, time_block=1)
    b = run_gpu(wl, steps, time_block=TB)
    assert a["info"]["time_block"] == 1 and b["info"]["time_block"] == 4
    for k in ("u", "v", "sigma"):
        assert np.array_equal(a[k], b[k]), (k, float(np.abs(a[k] - b[k]).max()))


@pytest.mark.parametrize("wl,steps", [(W.hole_plate(256, 128, 16.0, 0, lam_over_mu=0.8), 300),
                                      (_with(W.edge_crack(256, 64, 0, lam_over_mu=PAPER),
                                             wall_node=True), 300)],
                         ids=["hole_256x128_nonpoisson", "edge_crack_256_paper_node"])
def test_blocked_nonpoisson_parity_with_oracle(oracle_mod, wl, steps):
    gpu = run_gpu(wl, steps, time_block=TB)
    assert gpu["info"]["time_block"] == 4
    err = compare(gpu, run_oracle(oracle_mod, wl, steps))
    assert all(e <= 1e-5 for e in err.values()), err


def test_blocked_nonpoisson_full_size_crack_bit_identical():
    # the 2048^2 edge crack in the paper's material (nu = 0.2174) over 1500 steps
    wl = _with(W.CONFIG3, wall_node=True, lam_over_mu=PAPER)
    a = run_gpu(wl, wl.steps, time_block=1)
    b = run_gpu(wl, wl.steps, time_block=TB)
    for k in ("u", "v", "sigma"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("lam_over_mu", [1.0, 0.8], ids=["k_wave", "k_wave_grad"])
def test_wait_limit_runs_out_cleanly(lam_over_mu):
    """With a wait limit of 0 the blocked kernels give up on their first tile
    copy: every block stops before reading a ring row that has not landed,
    drains the copies it has in flight and exits, and the host sees
    LBM_ERR_TIMEOUT from lbm_sync and from the next lbm_step.  The context
    stays usable: with the default limit back and a reset, the same handle
    runs bit-identically to one step per launch."""
    wl = W.edge_crack(256, 64, 0, lam_over_mu=lam_over_mu)
    s = N.Solver(N.desc_from_workload(wl, time_block=TB))
    assert s.info()["time_block"] > 1
    N.lbm_set_wait_limit(s.h, 0)
    s.step(16)
    with pytest.raises(N.LbmError) as e:
        s.sync()
    assert e.value.status == N.LBM_ERR_TIMEOUT
    with pytest.raises(N.LbmError) as e:   # the next asynchronous call reports it too
        s.step(1)
        s.step(1)
    assert e.value.status == N.LBM_ERR_TIMEOUT
    with pytest.raises(N.LbmError) as e:
        N.lbm_set_wait_limit(s.h, -1)
    assert e.value.status == N.LBM_ERR_ARG
    N.lbm_set_wait_limit(s.h, 10 ** 9)
    s.reset()
    s.step(45)
    s.sync()
    got = s.fields_host()
    s.close()
    ref = run_gpu(wl, 45, time_block=1)
    for k in ("u", "v", "sigma"):
        assert np.array_equal(got[k], ref[k]), k
