"""The allocation-free fields entry point, lbm_get_fields_host_noalloc.

It serves callers that must not allocate device memory (a workspace sized up
front by another allocator, or a latency-critical path where cudaMalloc and its
implicit synchronisation are not acceptable): it stages the field planes in a
fixed array inside the library instead of the handle's workspace.  It runs the
same field kernels on the same state, so its output must equal what
lbm_get_fields returns bit for bit, call after call (host planes are filled
with NaN before each call, so a plane left unwritten fails), for both streaming
forms; lattices larger than the array must be refused.

This file is collected last so that a run stopping at the first failure has run
every other test before it.
"""
import numpy as np
import pytest

from paper_2208_04088_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _host_planes(ny, nx):
    return (np.full((2, ny, nx), np.nan, np.float32), np.full((2, ny, nx), np.nan, np.float32),
            np.full((3, ny, nx), np.nan, np.float32))


@pytest.mark.parametrize("wl,in_place", [(W.hole_plate(256, 128, 16.0, 0), False),
                                         (W.hole_plate(256, 128, 16.0, 0), True),
                                         (W.edge_crack(192, 50, 0,
                                                       lam_over_mu=W.CRACK_PAPER_LAM_OVER_MU), False),
                                         (W.square_plate(512, 0), False)],
                         ids=["hole_plate", "hole_plate_in_place", "crack_paper_material",
                              "square_512"])
def test_noalloc_fields_match_lbm_get_fields(wl, in_place):
    from paper_2208_04088_gb300 import _native as N
    s = N.Solver(N.desc_from_workload(wl, in_place=in_place))
    assert s.info()["streaming"] == (N.LBM_STREAM_IN_PLACE if in_place else
                                     N.LBM_STREAM_TWO_BUFFERS)
    for steps in (120, 35):
        s.step(steps)
        ref = s.fields_host()                       # the existing entry point
        assert np.abs(ref["sigma"]).max() > 0.0
        for _ in range(2):                          # two calls of the new one in a row
            u, v, sg = _host_planes(wl.ny, wl.nx)
            N.lbm_get_fields_host_noalloc(s.h, u.ctypes.data, v.ctypes.data, sg.ctypes.data)
            for name, got in (("u", u), ("v", v), ("sigma", sg)):
                assert np.array_equal(got, ref[name]), name
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
