"""GPU: in-place streaming (lbm_desc.streaming = LBM_STREAM_IN_PLACE).

One population buffer, updated in the AA pattern: even steps read and write
each node's own slots, odd steps the slots of its neighbours.  Boundary nodes
read all their inputs (their own and their upstream nodes' post-collision
populations) before any population is overwritten, then store.  The
arithmetic is that of the two-buffer form, so the fields must be
bit-identical to it after any number of steps, for every geometry and
storage, in one call or in chunks (replayed graphs and remainders of both
parities), and after a reset.
"""
import dataclasses

import numpy as np
import pytest

from paper_2208_04088_gb300 import _native as N
from paper_2208_04088_gb300 import workloads as W

from helpers import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _with(wl, **kw):
    return dataclasses.replace(wl, **kw)


def _moving_wall_plate():
    # Dirichlet edge with a ramped wall velocity and traction edges
    wl = W.square_plate(96, 0)
    wl.bcs = [W.bc(W.DIRICHLET, (2e-4, -1e-4), W.RAMP, 13.0), W.bc(W.TRACTION, (1e-3, 5e-4)),
              W.bc(W.TRACTION, (0.0, 0.0))]
    wl.name = "moving_wall_96"
    return wl


CASES = [
    _with(W.hole_plate(256, 128, 16.0, 0), name="hole_256x128_extrapolate"),
    _with(W.hole_plate(250, 130, 23.5, 0, profile=W.RAMP, t_ramp=17.0), wall_node=True,
          name="hole_ramp_250x130_node"),
    _with(W.square_plate(64, 0), name="square_64"),
    _moving_wall_plate(),
    _with(W.edge_crack(256, 64, 0), wall_node=True, name="edge_crack_256_L64_node"),
    _with(W.centre_crack(32, 0), name="centre_crack_128_L32"),
    # nearly every node a boundary node: the staging area is sized by the boundary list
    _with(W.square_plate(3, 0), name="square_3"),
    _with(W.square_plate(5, 0), name="square_5"),
]


def _same(a, b):
    for k in ("u", "v", "sigma"):
        assert np.array_equal(a[k], b[k]), (k, float(np.abs(a[k] - b[k]).max()))


@pytest.mark.parametrize("steps", [1, 2, 7, 40, 77])
@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_in_place_bit_identical_to_two_buffers(wl, steps):
    a = run_gpu(wl, steps, time_block=1)
    b = run_gpu(wl, steps, time_block=1, in_place=True)
    assert a["info"]["streaming"] == N.LBM_STREAM_TWO_BUFFERS
    assert b["info"]["streaming"] == N.LBM_STREAM_IN_PLACE
    _same(a, b)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("wl", [CASES[0], CASES[4]], ids=lambda w: w.name)
def test_in_place_bit_identical_16_bit(wl, storage):
    a = run_gpu(wl, 45, storage=storage)
    b = run_gpu(wl, 45, storage=storage, in_place=True)
    _same(a, b)


def test_in_place_in_chunks_and_after_reset():
    # odd and even chunk lengths: replayed graphs and direct launches of both parities
    wl = CASES[0]
    a = run_gpu(wl, 100, time_block=1)
    b = run_gpu(wl, 100, in_place=True, chunks=[3, 40, 9, 48])
    _same(a, b)
    d = N.desc_from_workload(wl, in_place=True)
    s = N.Solver(d)
    s.step(33)
    s.reset()
    s.step(100)
    s.sync()
    c = s.fields_host()
    s.close()
    _same(a, c)


def test_in_place_workspace_and_default_form():
    wl = W.edge_crack(2048, 512, 0)  # blocked by default with two buffers
    two = N.lbm_workspace_size(N.desc_from_workload(wl, time_block=1))
    one = N.lbm_workspace_size(N.desc_from_workload(wl, in_place=True))
    nx, ny = 2048, 2048
    # one buffer of 9 planes padded by a ring of one node, instead of two
    assert two - one > 9 * 4 * nx * ny * 0.9
    s = N.Solver(N.desc_from_workload(wl, in_place=True))
    info = s.info()
    s.close()
    assert info["time_block"] == 1 and info["streaming"] == N.LBM_STREAM_IN_PLACE


def test_in_place_parity_with_oracle(oracle_mod):
    wl = W.hole_plate(256, 128, 16.0, 0)
    gpu = run_gpu(wl, 500, in_place=True)
    err = compare(gpu, run_oracle(oracle_mod, wl, 500))
    assert all(e <= 1e-5 for e in err.values()), err
