"""Batched and served solves: many instances advanced by one persistent launch
per step must give every instance bit-identical fields to the same instance
stepped alone (the per-node code is shared), for every launch shape the
autotuner may pick, and with requests joining and leaving the server at
different times under a device-memory budget."""
import numpy as np
import pytest

from paper_2208_04088_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _alone(wl, steps, storage="f32"):
    from paper_2208_04088_gb300 import _native as N
    s = N.Solver(N.desc_from_workload(wl, storage=storage))
    s.step(steps)
    F = s.fields_host()
    s.close()
    return F


def _mix():
    return [W.hole_plate(256, 128, 16.0, 0), W.edge_crack(128, 32, 0),
            W.square_plate(64, 0), W.hole_plate(200, 96, 11.0, 0, load=4e-4),
            W.edge_crack(96, 24, 0, ny=64), W.square_plate(5, 0), W.hole_plate(77, 45, 9.5, 0)]


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("u", "v", "sigma"))


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_matches_instances_alone(storage):
    from paper_2208_04088_gb300 import _native as N
    wls = _mix()
    b = N.Batch([N.desc_from_workload(w, storage=storage) for w in wls])
    b.step(75)                 # four replayed 16-step graphs and 11 direct steps
    b.sync()
    for k, w in enumerate(wls):
        assert _same(b.fields_host(k), _alone(w, 75, storage)), w.name
    info = b.info()
    assert info["instances"] == len(wls) and info["steps"] == 75
    b.close()


def test_blocked_batch_across_buffer_parities():
    """Instances of at least 128 columns in FP32 take the temporally blocked
    batch kernel.  Calls of 37, 16 and 27 steps replay chunks that start in
    either population buffer (a chunk after an odd remainder) and finish with
    the instances' own blocked and one-step launches; every instance stays
    bit-identical to itself stepped alone, at every call boundary."""
    from paper_2208_04088_gb300 import _native as N
    wls = [W.hole_plate(300, 140, 23.5, 0), W.edge_crack(256, 64, 0, ny=96),
           W.square_plate(128, 0), W.hole_plate(128, 64, 8.0, 0), W.hole_plate(96, 64, 9.0, 0)]
    b = N.Batch([N.desc_from_workload(w) for w in wls])
    assert b.info()["blocked_instances"] == 4
    t = 0
    for n in (37, 16, 27):
        b.step(n)
        t += n
        for k, w in enumerate(wls):
            assert _same(b.fields_host(k), _alone(w, t)), (t, w.name)
    b.reset()
    b.step(16)
    for k, w in enumerate(wls):
        assert _same(b.fields_host(k), _alone(w, 16)), ("after reset", w.name)
    b.close()


def test_every_launch_shape_and_the_tuner_give_identical_fields():
    from paper_2208_04088_gb300 import _native as N
    wls = _mix()
    ref = [_alone(w, 40) for w in wls]
    b = N.Batch([N.desc_from_workload(w) for w in wls])
    for shape in [(32, 8, 8, 0), (32, 8, 4, 1), (32, 4, 16, 0), (64, 4, 8, 1), (32, 16, 4, 0),
                  (32, 4, 16, 3), (64, 4, 8, 3)]:
        b.reset()
        b.set_shape(*shape)
        b.step(40)
        for k in range(len(wls)):
            assert _same(b.fields_host(k), ref[k]), (shape, wls[k].name)
    chosen = b.tune(steps_per_trial=8)   # leaves every instance at rest, t = 0
    assert chosen["tile_x"] in (32, 64)
    b.step(40)
    for k in range(len(wls)):
        assert _same(b.fields_host(k), ref[k])
    b.close()


def test_server_results_equal_alone_with_joins_and_budget():
    from paper_2208_04088_gb300 import _native as N
    reqs = [(W.hole_plate(256, 128, 16.0, 0), 90), (W.edge_crack(128, 32, 0), 37),
            (W.square_plate(64, 0), 150), (W.hole_plate(77, 45, 9.5, 0), 20),
            (W.edge_crack(96, 24, 0, ny=64), 64), (W.square_plate(48, 0), 5)]
    # a budget that holds the first request but not all of them at once
    budget = N.lbm_workspace_size(N.desc_from_workload(reqs[0][0])) * 3 // 2
    srv = N.Server(budget)
    ids = []
    results = {}
    pending = list(reqs)
    ticks = 0
    while len(results) < len(reqs):
        # one new request arrives every other tick, while earlier ones run
        if pending and ticks % 2 == 0:
            w, n = pending.pop(0)
            ids.append((srv.submit(N.desc_from_workload(w), n), w, n))
        st = srv.tick(max_steps=16)
        assert st["device_bytes"] <= budget
        for rid, w, n in ids:
            if rid in results:
                continue
            r = srv.result(rid)
            if r is not None:
                results[rid] = (r, w, n)
        ticks += 1
        assert ticks < 500
    for rid, (r, w, n) in results.items():
        assert _same(r, _alone(w, n)), (w.name, n)
    srv.close()


def test_server_rejects_requests_it_cannot_run():
    from paper_2208_04088_gb300 import _native as N
    srv = N.Server(64 << 20)
    big = N.desc_from_workload(W.square_plate(2048, 0))       # > 64 MiB workspace
    with pytest.raises(N.LbmError) as e:
        srv.submit(big, 10)
    assert e.value.status == N.LBM_ERR_NOMEM
    # lambda != mu needs the density pass of the single-solver path
    rid = srv.submit(N.desc_from_workload(W.square_plate(32, 0, lam_over_mu=0.8)), 10)
    srv.tick(8)
    with pytest.raises(N.LbmError):
        srv.result(rid)
    srv.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_in_place_instances_match_alone(storage):
    """Instances with in-place streaming, alone or mixed with two-buffer ones,
    give the fields of the two-buffer solver run alone."""
    from paper_2208_04088_gb300 import _native as N
    wls = _mix()
    ref = [_alone(w, 75, storage) for w in wls]
    for mixed in (False, True):
        descs = [N.desc_from_workload(w, storage=storage, in_place=not mixed or k % 2 == 0)
                 for k, w in enumerate(wls)]
        b = N.Batch(descs)
        b.step(75)
        b.sync()
        for k, w in enumerate(wls):
            assert _same(b.fields_host(k), ref[k]), (mixed, w.name)
        for shape in [(32, 4, 16, 0), (64, 4, 8, 1), (32, 8, 8, 3)]:
            b.reset()
            b.set_shape(*shape)
            b.step(75)
            for k in range(len(wls)):
                assert _same(b.fields_host(k), ref[k]), (mixed, shape, wls[k].name)
        b.close()


def test_server_in_place_requests_join_at_any_parity():
    """In-place requests joining a running server at odd and even times of the
    others (each instance keeps its own clock and parity) end with the fields
    they have alone; they also need less of the budget."""
    from paper_2208_04088_gb300 import _native as N
    reqs = [(W.hole_plate(256, 128, 16.0, 0), 90, True), (W.edge_crack(128, 32, 0), 37, False),
            (W.square_plate(64, 0), 151, True), (W.hole_plate(77, 45, 9.5, 0), 21, True),
            (W.edge_crack(96, 24, 0, ny=64), 64, False), (W.square_plate(48, 0), 5, True)]
    w0 = reqs[0][0]
    assert N.lbm_workspace_size(N.desc_from_workload(w0, in_place=True)) < \
        N.lbm_workspace_size(N.desc_from_workload(w0))
    srv = N.Server(N.lbm_workspace_size(N.desc_from_workload(w0)) * 3)
    ids, results, pending, ticks = [], {}, list(reqs), 0
    while len(results) < len(reqs):
        if pending and ticks % 2 == 0:
            w, n, ip = pending.pop(0)
            ids.append((srv.submit(N.desc_from_workload(w, in_place=ip), n), w, n))
        srv.tick(max_steps=7)  # odd ticks: requests join at odd and even times of the others
        for rid, w, n in ids:
            if rid not in results:
                r = srv.result(rid)
                if r is not None:
                    results[rid] = (r, w, n)
        ticks += 1
        assert ticks < 500
    for rid, (r, w, n) in results.items():
        assert _same(r, _alone(w, n)), (w.name, n)
    srv.close()
