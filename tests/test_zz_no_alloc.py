"""The allocation-free fields entry point, lbm_get_fields_host_noalloc.

It serves callers that must not allocate device memory (a workspace sized up
front by another allocator, or a latency-critical path where cudaMalloc and its
implicit synchronisation are not acceptable): it stages the field planes in a
fixed array inside the library instead of the handle's workspace.  Its output
must equal what lbm_get_fields returns, call after call, and lattices larger
than the array must be refused.

This file is collected last so that a run stopping at the first failure has run
every other test before it.
"""
import numpy as np
import pytest

from paper_2208_04088_gb300 import workloads as W

from helpers import rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _host_planes(ny, nx):
    return (np.empty((2, ny, nx), np.float32), np.empty((2, ny, nx), np.float32),
            np.empty((3, ny, nx), np.float32))


@pytest.mark.parametrize("wl", [W.hole_plate(256, 128, 16.0, 0),
                                W.edge_crack(192, 50, 0, lam_over_mu=W.CRACK_PAPER_LAM_OVER_MU),
                                W.square_plate(512, 0)],
                         ids=lambda w: w.name)
def test_noalloc_fields_match_lbm_get_fields(wl):
    from paper_2208_04088_gb300 import _native as N
    s = N.Solver(N.desc_from_workload(wl))
    mask = np.ones((wl.ny, wl.nx), dtype=bool)
    for steps in (120, 35):
        s.step(steps)
        ref = s.fields_host()                       # the existing entry point
        for _ in range(2):                          # two calls of the new one in a row
            u, v, sg = _host_planes(wl.ny, wl.nx)
            N.lbm_get_fields_host_noalloc(s.h, u.ctypes.data, v.ctypes.data, sg.ctypes.data)
            for name, got in (("u", u), ("v", v), ("sigma", sg)):
                err = rel_l2(got, ref[name], mask)
                assert err <= TOL, (name, err)
    s.close()


def test_noalloc_rejects_lattices_beyond_the_static_array():
    from paper_2208_04088_gb300 import _native as N
    wl = W.square_plate(600, 0)                     # 360000 nodes > 262144
    s = N.Solver(N.desc_from_workload(wl))
    u, v, sg = _host_planes(wl.ny, wl.nx)
    with pytest.raises(N.LbmError) as e:
        N.lbm_get_fields_host_noalloc(s.h, u.ctypes.data, v.ctypes.data, sg.ctypes.data)
    assert e.value.status == N.LBM_ERR_ARG
    assert "262144" in str(e.value)
    s.close()
