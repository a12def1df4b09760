"""Serving scheduler host logic (CPU): admission policy and refusal without any GPU work."""
import numpy as np

from paper_2604_09643_b300 import serve, synth


def test_admission_policy():
    GB = 1 << 30
    assert serve.admission(10 * GB, 100 * GB, 200 * GB, 2 * GB) == serve.ADMIT
    assert serve.admission(10 * GB, 11 * GB, 200 * GB, 2 * GB) == serve.WAIT
    assert serve.admission(199 * GB, 200 * GB, 200 * GB, 2 * GB) == serve.REJECT


def test_footprint_grows_with_the_scan():
    small = synth.make_geom((64, 64, 64), 0.1, 64, 16, 1024)
    big = synth.make_geom((256, 256, 256), 0.1, 1024, 256, 3072)
    assert 0 < serve.footprint_bytes(small) < serve.footprint_bytes(big)


def _req(i, n=32, F=4):
    geom = synth.make_geom((n, n, n), 0.2, 16, F, 256)
    return serve.Request(i, 0.0, geom, synth.planar_array(4, 4, 0.5),
                         np.zeros((F, 16, 256), np.float32), np.tile(np.eye(3, 4), (F, 1, 1)), steps=2)


def test_oversize_request_is_refused_with_a_status():
    GB = 1 << 30
    srv = serve.Server(device=0, reserve_bytes=0, mem_info=lambda: (GB // 1024, GB // 1024))
    srv.submit(_req(0))
    res = srv.run(max_seconds=1.0)
    assert len(res) == 1 and res[0].status.startswith("rejected")


def test_request_that_does_not_fit_with_nothing_running_is_refused():
    """Waiting only helps while running scans can release memory: with none running
    the request is refused with a status instead of waiting forever."""
    GB = 1 << 30
    srv = serve.Server(device=0, reserve_bytes=0, mem_info=lambda: (0, 100 * GB))
    srv.submit(_req(0))
    res = srv.run()
    assert len(res) == 1 and res[0].status.startswith("rejected") and "no scan running" in res[0].status
    assert not srv.queue


def test_iteration_work_cap_holds_requests_until_the_iteration_has_room(monkeypatch):
    """With max_iteration_pairs, a request that would take the resident scans' pairs per
    step past the cap waits (FIFO) while others run; with nothing running it is admitted
    whatever its size.  Host logic only: scans are stand-ins."""
    GB = 1 << 30
    admitted = []

    class FakeScan:
        def __init__(self, req, device, now, stream=None):
            self.req = req
            admitted.append(req.id)

    monkeypatch.setattr(serve, "_Scan", FakeScan)
    srv = serve.Server(device=0, reserve_bytes=0, mem_info=lambda: (100 * GB, 100 * GB),
                       max_iteration_pairs=2 * serve.step_pairs(_req(0).geom))
    srv._stream = object()  # no device stream needed for admission
    srv.t0 = srv.clock()
    for i in range(4):
        srv.submit(_req(i))
    srv._admit()
    assert admitted == [0, 1] and [r.id for r in srv.queue] == [2, 3]
    srv.active = []          # the resident scans finished
    srv.max_iteration_pairs = 1   # smaller than any scan: admitted only into an empty iteration
    srv._admit()
    assert admitted == [0, 1, 2] and [r.id for r in srv.queue] == [3]


def test_fair_share_fills_the_iteration_with_the_least_served_scans():
    """The next batched iteration takes scans by pairs served so far (then arrival), first
    fit into the budget; the least-served is always taken, even when it alone exceeds it."""
    class S:
        def __init__(self, i, n, served):
            self.req = _req(i, n=n)
            self.served_pairs = served

    small = [S(0, 16, 0), S(1, 16, 10), S(2, 16, 5)]
    big = S(3, 64, 1)
    per_small = serve.step_pairs(small[0].req.geom)
    pick = serve.fair_share(small + [big], 2 * per_small)
    assert [x.req.id for x in pick] == [0, 2]            # least served first; the big one does not fit
    pick = serve.fair_share([big, small[1]], per_small)  # the big one is the least served: alone
    assert [x.req.id for x in pick] == [3]
    pick = serve.fair_share(small, 10 ** 15)
    assert sorted(x.req.id for x in pick) == [0, 1, 2]
