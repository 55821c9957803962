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


# ------------------------------------------------------------------ stepped engine
class FakeStepServer(S.Server):
    """The stepped engine with simulated solves: a request of `cycles` restart cycles,
    each taking `dt` seconds; no device work."""

    def __init__(self, *a, **kw):
        self.starts, self.finish_order = [], []
        self.lock2 = threading.Lock()
        super().__init__(*a, **kw)

    def footprint_of(self, req, R=4):
        return req.problem.bytes

    def _start_unit(self, unit):
        if any(getattr(r.problem, "fail", False) for r in unit.group):
            raise ValueError("plan creation failed")
        with self.lock2:
            self.starts.append([r.rid for r in unit.group])
        unit.cycles = 1
        unit.solver = 1
        unit.t_ready = time.perf_counter() + unit.group[0].problem.dt
        unit.need_cycles = max(r.problem.cycles for r in unit.group)

    def _state(self, unit):
        if time.perf_counter() < unit.t_ready:
            return ie.IE_SOLVER_BUSY, {}
        if unit.cycles >= unit.need_cycles:
            return ie.IE_SOLVER_DONE, {"converged": 1, "iterations": 50 * unit.cycles}
        return ie.IE_SOLVER_IDLE, {"converged": 0}

    def _advance(self, unit):
        unit.cycles += 1
        unit.t_ready = time.perf_counter() + unit.group[0].problem.dt

    def _harvest(self, unit, st, info):
        with self.lock2:
            self.finish_order.append([r.rid for r in unit.group])
        for r in unit.group:
            r.status, r.info = st, dict(info)

    def _teardown(self, unit):
        unit.solver = 0


def _sreq(rid, nbytes, cycles, dt=0.01, G=16, fail=False):
    prob = SimpleNamespace(G=G, bytes=nbytes, nb=np.full(4, 32, dtype=np.int32), cycles=cycles, dt=dt, fail=fail)
    return S.Request(rid=rid, problem=prob, khat=np.zeros((1, 3)), pol=np.zeros((1, 3)))


def _step_server(**kw):
    opts = ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X3, restart=50, max_iters=500)
    return FakeStepServer([ie.IE_PREC_FP16X3], opts, **kw)


def test_stepped_short_request_overtakes_a_long_one():
    """One builder thread: a short solve submitted while a long one runs starts at once
    and finishes first (no head-of-line blocking behind a running solve)."""
    srv = _step_server(budget=100, workers=1)
    assert srv.stepped
    try:
        srv.submit(_sreq(0, 10, cycles=8, dt=0.05))
        time.sleep(0.06)
        srv.submit(_sreq(1, 10, cycles=1, dt=0.01))
        done = srv.drain(2, timeout=30)
    finally:
        srv.close()
    assert srv.finish_order == [[1], [0]]
    by = {r.rid: r for r in done}
    assert by[1].t_done < by[0].t_done and all(r.status == ie.IE_OK for r in done)
    assert srv.max_live == 2


def test_stepped_budget_bounds_live_solves():
    srv = _step_server(budget=100, workers=4)
    try:
        for i in range(8):
            srv.submit(_sreq(i, 40, cycles=2))
        done = srv.drain(8, timeout=30)
    finally:
        srv.close()
    assert srv.peak_used <= 100 and srv.max_live <= 2
    assert sorted(r.rid for r in done) == list(range(8)) and srv.used == 0


def test_stepped_cycle_cap_and_failures():
    """A solve still iterating after max_iters / restart + 2 cycles is reported as not
    converged; a unit whose set-up fails reports its error and gives its memory back."""
    srv = _step_server(budget=100, workers=2)
    try:
        srv.submit(_sreq(0, 10, cycles=10 ** 6, dt=0.001))
        srv.submit(_sreq(1, 10, cycles=1, fail=True))
        done = srv.drain(2, timeout=30)
    finally:
        srv.close()
    by = {r.rid: r for r in done}
    assert by[0].status == ie.IE_ERR_NOT_CONVERGED
    assert "plan creation failed" in by[1].error and srv.used == 0
