"""Host logic of the serving scheduler (no GPU): FIFO admission by device
footprint, the memory budget, batching of queued requests on one grid."""
import threading
import time
from types import SimpleNamespace

import numpy as np

import paper_2501_04684_gb300 as ie
from paper_2501_04684_gb300 import serve as S


class FakeServer(S.Server):
    """Runs no device work: each unit of work sleeps and records what ran together."""

    def __init__(self, *a, **kw):
        self.log = []
        self.active = 0
        self.max_active = 0
        self.lock = threading.Lock()
        super().__init__(*a, **kw)

    def footprint_of(self, req, R=4):
        return req.problem.bytes

    def _run(self, group, stream):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.log.append([r.rid for r in group])
        time.sleep(0.02)
        for r in group:
            r.status = ie.IE_OK
        with self.lock:
            self.active -= 1


def _req(rid, nbytes, G=16):
    prob = SimpleNamespace(G=G, bytes=nbytes, nb=np.full(4, 32, dtype=np.int32))
    return S.Request(rid=rid, problem=prob, khat=np.zeros((1, 3)), pol=np.zeros((1, 3)))


def _serve(reqs, **kw):
    srv = FakeServer([ie.IE_PREC_FP32], None, **kw)
    try:
        for r in reqs:
            srv.submit(r)
        done = srv.drain(len(reqs), timeout=30)
    finally:
        srv.close()
    return srv, done


def test_fifo_single_worker():
    srv, done = _serve([_req(i, 10) for i in range(6)], budget=100, workers=1)
    assert [g[0] for g in srv.log] == list(range(6))
    assert all(r.status == ie.IE_OK and r.latency >= 0 for r in done)


def test_budget_bounds_concurrency():
    srv, _ = _serve([_req(i, 40) for i in range(8)], budget=100, workers=4)
    assert srv.peak_used <= 100
    assert srv.max_active <= 2          # two 40-byte requests fit a 100-byte budget


def test_oversized_request_runs_alone():
    reqs = [_req(0, 10), _req(1, 500), _req(2, 10)]
    srv, done = _serve(reqs, budget=100, workers=3)
    assert len(done) == 3
    assert sorted(g[0] for g in srv.log) == [0, 1, 2]


def test_batching_merges_same_grid_only():
    reqs = [_req(0, 10, G=16), _req(1, 10, G=32), _req(2, 10, G=16), _req(3, 10, G=16), _req(4, 10, G=32)]
    srv = FakeServer([ie.IE_PREC_FP32], None, budget=1000, workers=1, batch=3)
    # hold the worker until every request is queued, so batches can form
    with srv.cv:
        for r in reqs:
            r.footprint = 10
            r.t_submit = srv.now()
            srv.queue.append(r)
        srv.cv.notify_all()
    srv.drain(5, timeout=30)
    srv.close()
    assert srv.log[0] == [0, 2, 3]
    assert srv.log[1] == [1, 4]
