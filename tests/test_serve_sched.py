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


# ------------------------------------------------------------------ shared stores
class _FakeStore:
    """Stands in for ie.Store (no device memory): keeps its spec and a byte count."""

    def __init__(self, spec):
        self.spec = spec
        self.info = {"bytes": 1000 * spec.max_disp}
        self.closed = False

    def close(self):
        self.closed = True


def _reach_problem(reach, k=1.0):
    return SimpleNamespace(k=k, eta=2.0, a=0.25, box_ijk=np.array([[0, 0, 0], [reach, 1, 0]]))


def test_shared_store_grows_in_steps_of_eight_and_counts_against_the_budget(monkeypatch):
    """One store per (k, eta, a), reused while it reaches far enough, replaced by one of
    larger reach (rounded up to a multiple of 8 boxes) when a scatterer reaches farther;
    every store made counts against the budget (a replaced one may still be held by
    plans attached to it)."""
    monkeypatch.setattr(S.ie, "Store", _FakeStore)
    srv = S.Server([ie.IE_PREC_FP16X3], None, budget=10 ** 9, workers=1, symmetry=1)
    try:
        assert srv.share
        s1 = srv.store_for(_reach_problem(5))
        assert s1.spec.max_disp == 8 and srv.store_bytes == srv.used == 8000
        assert srv.store_for(_reach_problem(8)) is s1
        s2 = srv.store_for(_reach_problem(9))
        assert s2.spec.max_disp == 16 and s1.closed and not s2.closed
        assert srv.store_bytes == srv.used == 8000 + 16000 and srv.peak_used == 24000
        s3 = srv.store_for(_reach_problem(3, k=2.0))
        assert s3 is not s2 and s3.spec.max_disp == 8 and len(srv.stores) == 2
    finally:
        srv.close()
    assert s2.closed and s3.closed and not srv.stores


def test_prepare_stores_makes_one_store_of_the_largest_reach(monkeypatch):
    monkeypatch.setattr(S.ie, "Store", _FakeStore)
    srv = S.Server([ie.IE_PREC_FP16X3], None, budget=10 ** 9, workers=1, symmetry=1)
    try:
        srv.prepare_stores([_reach_problem(r) for r in (4, 17, 9)])
        (st,) = srv.stores.values()
        assert st.spec.max_disp == 24
        assert srv.store_for(_reach_problem(17)) is st
    finally:
        srv.close()
