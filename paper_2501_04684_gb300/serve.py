"""Continuous serving of scattering solves on one GPU over the C ABI.

Requests (one scatterer, 1-4 plane-wave excitations each) arrive over time.  The
scheduler admits them in arrival order while their device footprint fits the HBM
budget.  With `batch` > 1 the requests queued behind the head that share its grid are
merged into one batched plan (independent scatterers in one plan, one launch per
kernel) and solved together.

Coupling blocks: the far translations depend on k, eta, the box edge and the sorted
|d| only (end of §2, §2.2), so with symmetry = 1 every plan attaches to one shared
store per (k, eta, box edge) - generated once, outside any request's latency, and
grown (a new store of larger reach) when a scatterer reaches farther than the current
one - and builds only its pair lists and near blocks.

Two ways of running admitted work:
  stepped (opts without refinement; the default then): builder threads make the plan,
    the excitation and a solver object and enqueue its first restart cycle (one unit's
    set-up at a time: allocation and graph capture never overlap another's); one engine
    thread then advances every live solve one GMRES(m) cycle at a time on its own stream
    (ie_solver_advance, ie_solver_state read from pinned memory, no host
    synchronisation), so a request admitted while others run starts at once and runs
    beside them instead of waiting for a worker; finished solves go to a reaper thread
    that tears them down.
  blocking (refinement, or stepped=False): each admitted unit runs ie_solve on a worker
    thread and stream.
Every device step runs in libie; this module only orders the calls.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

import paper_2501_04684_gb300 as ie


@dataclass
class Request:
    """One scattering solve: a scatterer and its plane waves."""
    rid: int
    problem: object          # workloads.Problem-like: G, box_ijk, nb, P, alpha, k, eta, a, lattice
    khat: np.ndarray         # (nrhs, 3)
    pol: np.ndarray          # (nrhs, 3)
    t_submit: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    info: dict = field(default_factory=dict)
    status: int = -1
    error: str = ""
    x: object = None         # solution tensor [nrhs][n] (kept only with keep_solutions)
    footprint: int = 0       # device bytes reserved for it (computed at submission when 0)

    @property
    def nrhs(self) -> int:
        return int(np.asarray(self.khat).reshape(-1, 3).shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


class _BatchView:
    """Members of a merged batch in the form problem_from_batch takes."""

    def __init__(self, reqs):
        self.members = [r.problem for r in reqs]
        self.G = reqs[0].problem.G
        self.R = max(r.nrhs for r in reqs)
        self.nrhs = [r.nrhs for r in reqs]

    box_ijk = property(lambda s: np.concatenate([m.box_ijk for m in s.members]).astype(np.int32))
    nb = property(lambda s: np.concatenate([m.nb for m in s.members]).astype(np.int32))
    P = property(lambda s: np.concatenate([m.P for m in s.members]))
    box_group = property(lambda s: np.concatenate([np.full(m.box_ijk.shape[0], g, dtype=np.int32)
                                                   for g, m in enumerate(s.members)]))
    group_alpha = property(lambda s: np.array([m.alpha for m in s.members], dtype=np.float64))
    max_rhs = property(lambda s: s.R)


@dataclass
class _Unit:
    """Admitted work: one plan (one request, or a merged batch) and its solve."""
    group: list
    need: int
    stream: object = None
    plan: object = None
    solver: int = 0
    v: object = None
    x: object = None
    R: int = 1
    cycles: int = 0
    t_start: float = 0.0
    status: int = -1
    info: dict = field(default_factory=dict)
    error: str = ""


class Server:
    """FIFO admission by device footprint; stepped or blocking execution (module doc).

    precs / opts: the plan's precisions and the ie_solve options of every request.
    budget: device bytes the server may hold at once (shared stores included).
    workers: builder threads (stepped) or solve threads (blocking).  batch: most
    requests merged into one plan (same grid only).  keep_solutions: keep each
    request's solution.  symmetry: 1 builds symmetry-compressed plans (one coupling
    block per sorted |d|).  share_store: attach those plans to shared stores (default:
    with symmetry = 1).  stepped: None = stepped when opts has no refinement.
    streams: CUDA streams the stepped engine spreads live solves over.
    """

    def __init__(self, precs, opts, budget: int, workers: int = 4, batch: int = 1, keep_solutions: bool = False,
                 symmetry: int = 0, share_store: bool | None = None, stepped: bool | None = None, streams: int = 4):
        import torch
        self.torch = torch
        self.precs = list(precs)
        self.mask = ie.precmask(*precs)
        self.opts = opts
        self.budget = int(budget)
        self.batch = max(1, int(batch))
        self.keep = keep_solutions
        self.symmetry = int(symmetry)
        self.share = (self.symmetry == 1) if share_store is None else bool(share_store) and self.symmetry == 1
        refine = bool(getattr(opts, "refine", 0)) if opts is not None else True
        self.stepped = (not refine) if stepped is None else bool(stepped) and not refine
        self.queue: collections.deque = collections.deque()
        self.done: list = []
        self.used = 0
        self.cv = threading.Condition()
        self.closing = False
        self.t0 = time.perf_counter()
        self.peak_used = 0
        self.max_live = 0
        self.stores: dict = {}          # (k, eta, a) -> ie.Store of the largest reach so far
        self.store_lock = threading.Lock()
        self.store_bytes = 0
        self.live: list = []          # stepped: units the engine advances
        self.reap: collections.deque = collections.deque()
        self.building = 0
        self.setup_lock = threading.Lock()
        self.device = torch.cuda.current_device() if torch.cuda.is_available() else None
        self._streams = []
        if self.device is not None and self.stepped:
            self._streams = [torch.cuda.Stream() for _ in range(max(1, streams))]
        self._next_stream = 0
        target = self._builder if self.stepped else self._worker
        self.workers = [threading.Thread(target=target, daemon=True) for _ in range(workers)]
        self.engine = threading.Thread(target=self._engine, daemon=True) if self.stepped else None
        self.reaper = threading.Thread(target=self._reaper, daemon=True) if self.stepped else None
        for t in self.workers + [t for t in (self.engine, self.reaper) if t is not None]:
            t.start()

    # ---------------------------------------------------------------- client side
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        if not req.footprint:
            req.footprint = self.footprint_of(req, 4 if self.batch > 1 else req.nrhs)
        with self.cv:
            req.t_submit = self.now()
            self.queue.append(req)
            self.cv.notify_all()

    def drain(self, count: int, timeout: float = 3600.0):
        """Wait until `count` requests have completed."""
        end = time.perf_counter() + timeout
        with self.cv:
            while len(self.done) < count:
                left = end - time.perf_counter()
                if left <= 0:
                    raise TimeoutError(f"{len(self.done)} of {count} requests done")
                self.cv.wait(min(left, 1.0))
        return list(self.done)

    def close(self):
        with self.cv:
            self.closing = True
            self.cv.notify_all()
        for t in self.workers + [t for t in (self.engine, self.reaper) if t is not None]:
            t.join()
        for st in self.stores.values():
            st.close()
        self.stores.clear()

    # ---------------------------------------------------------------- shared stores
    def prepare_stores(self, problems):
        """Create the shared stores for these scatterers ahead of their requests: one per
        (k, eta, box edge), of the largest reach among them."""
        if not self.share:
            return
        need = {}
        for p in problems:
            key = (float(p.k), float(p.eta), float(p.a))
            need[key] = max(need.get(key, 0), ie.max_far_disp(p.box_ijk))
        for (k, eta, a), reach in need.items():
            self.store_for(collections.namedtuple("Reach", "k eta a box_ijk")(k, eta, a, None), reach)

    def store_for(self, problem, reach: int | None = None):
        """The shared store serving `problem` (created, or replaced by one of larger reach,
        on demand; its bytes count against the budget from then on)."""
        key = (float(problem.k), float(problem.eta), float(problem.a))
        reach = ie.max_far_disp(problem.box_ijk) if reach is None else int(reach)
        with self.store_lock:
            st = self.stores.get(key)
            if st is not None and st.spec.max_disp >= reach:
                return st
            reach = max(reach, st.spec.max_disp if st is not None else 0)
            reach = max(2, int(math.ceil(reach / 8.0)) * 8)      # grow in steps of 8 boxes
            spec = ie.store_spec(key[0], key[1], key[2], reach, self.mask)
            new = ie.Store(spec)
            if st is not None:
                st.close()            # plans attached to it keep their reference
            self.stores[key] = new
            with self.cv:
                self.store_bytes += new.info["bytes"]
                self.used += new.info["bytes"]
                self.peak_used = max(self.peak_used, self.used)
            return new

    # ---------------------------------------------------------------- scheduler
    def footprint_of(self, req: Request, R: int = 4) -> int:
        """Device bytes of `req` in a plan of R columns (R >= its own nrhs): the plan
        (ie_plan_footprint, or ie_plan_footprint_shared without the store's blocks), the
        GMRES state, the refinement vectors and v, x.  Members of a merged plan share its
        coupling store, so a batch needs at most the sum of its members' footprints."""
        R = max(R, req.nrhs)
        n = int(req.problem.nb.sum())
        pr = ie.problem_from(req.problem, self.mask, R, symmetry=self.symmetry)
        if self.share:
            plan_b = ie.ie_plan_footprint_shared(pr, self.store_for(req.problem).handle)
        else:
            plan_b = ie.ie_plan_footprint(pr)
        m = self.opts.restart
        solver_b = (m + 3) * R * n * 8 + 64 * (m + 2) ** 2 * R
        refine_b = 4 * R * n * 16 if self.opts.refine else 0
        return plan_b + solver_b + refine_b + 2 * R * n * 8

    def _take(self):
        """Next unit of work that fits the budget (called with the lock held): the
        head of the queue, plus (batch > 1) queued requests on the head's grid."""
        if not self.queue:
            return None, 0
        head = self.queue[0]
        group = [head]
        if self.batch > 1:
            for r in list(self.queue)[1:]:
                if len(group) >= self.batch:
                    break
                if r.problem.G == head.problem.G:
                    group.append(r)
        while group:
            need = sum(r.footprint for r in group)
            if self.used + need <= self.budget or (self.used - self.store_bytes <= 0 and len(group) == 1):
                for r in group:
                    self.queue.remove(r)
                return group, need
            if len(group) == 1:
                return None, 0          # head-of-line waits for memory
            group.pop()
        return None, 0

    def _admit(self, building: bool = False):
        """Block until a unit is admitted (returns it) or the server closes (None).
        building: count it as being built (stepped mode) in the same critical section,
        so the engine never sees an empty server while a unit is on its way."""
        with self.cv:
            while True:
                if self.closing and not self.queue:
                    return None
                group, need = self._take()
                if group:
                    self.used += need
                    self.peak_used = max(self.peak_used, self.used)
                    if building:
                        self.building += 1
                    return _Unit(group=group, need=need, t_start=self.now())
                self.cv.wait(0.05)

    def _complete(self, unit: _Unit):
        """Record the unit's requests as done and give its memory back."""
        t_done = self.now()
        with self.cv:
            self.used -= unit.need
            for r in unit.group:
                r.t_start, r.t_done = unit.t_start, t_done
                if unit.error:
                    r.error = unit.error
                self.done.append(r)
            self.cv.notify_all()

    def _problem(self, unit: _Unit):
        """The plan's problem and the excitation of a unit."""
        group = unit.group
        if len(group) == 1:
            r = group[0]
            pr = ie.problem_from(r.problem, self.mask, r.nrhs, symmetry=self.symmetry)
            return pr, r.khat, r.pol, r.nrhs
        view = _BatchView(group)
        pr = ie.problem_from_batch(view, self.mask, symmetry=self.symmetry, exact_rhs=True)
        R = view.R
        khat = np.zeros((len(group), R, 3))
        khat[:, :, 2] = 1.0
        pol = np.zeros((len(group), R, 3))
        for g, r in enumerate(group):
            khat[g, :r.nrhs] = np.asarray(r.khat).reshape(-1, 3)
            pol[g, :r.nrhs] = np.asarray(r.pol).reshape(-1, 3)
        return pr, khat, pol, R

    def _make_plan(self, unit: _Unit, pr, stream):
        store = self.store_for(unit.group[0].problem) if self.share else None
        return ie.Plan(pr, stream, store=store)

    def _harvest(self, unit: _Unit, st: int, info: dict):
        """Status, info and (keep_solutions) solution slices of every request of a unit."""
        off = 0
        for r in unit.group:
            nr = int(r.problem.nb.sum())
            r.status, r.info = st, dict(info)
            if self.keep:
                r.x = unit.x[:r.nrhs, off:off + nr].clone()
            off += nr

    # ---------------------------------------------------------------- blocking mode
    def _worker(self):
        torch = self.torch
        stream = None
        if self.device is not None:
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream()
        while True:
            unit = self._admit()
            if unit is None:
                return
            try:
                self._run(unit.group, stream)
            except Exception as e:   # the request fails; the server keeps serving
                unit.error = f"{type(e).__name__}: {e}"
            self._complete(unit)

    def _run(self, group, stream):
        torch = self.torch
        unit = _Unit(group=group, need=0)
        with torch.cuda.stream(stream):
            pr, khat, pol, R = self._problem(unit)
            plan = self._make_plan(unit, pr, stream)
            try:
                unit.x = torch.zeros((R, plan.n), dtype=torch.complex64, device="cuda")
                v = torch.zeros_like(unit.x)
                ie.ie_rhs_plane_wave(plan.handle, khat, pol, v, stream)
                st, info = ie.ie_solve(plan.handle, v, unit.x, R, self.opts, stream)
                stream.synchronize()
                self._harvest(unit, st, info)
                del v
            finally:
                unit.x = None
                plan.close()

    # ---------------------------------------------------------------- stepped mode
    def _builder(self):
        """Admit units and make each one ready to step: plan, excitation, solver, start,
        first cycle enqueued; then hand it to the engine."""
        if self.device is not None:
            self.torch.cuda.set_device(self.device)
        while True:
            unit = self._admit(building=True)
            if unit is None:
                return
            with self.cv:
                unit.stream = self._streams[self._next_stream % len(self._streams)] if self._streams else None
                self._next_stream += 1
            try:
                with self.setup_lock:     # one unit's device set-up (allocation, capture) at a time
                    self._start_unit(unit)
                with self.cv:
                    self.live.append(unit)
                    self.max_live = max(self.max_live, len(self.live))
                    self.building -= 1
                    self.cv.notify_all()
            except Exception as e:
                unit.error = f"{type(e).__name__}: {e}"
                for r in unit.group:
                    r.status = ie.IE_ERR_INVALID if isinstance(e, (ValueError, ie.IEError)) else -1
                with self.cv:
                    self.building -= 1
                self._teardown(unit)
                self._complete(unit)

    def _start_unit(self, unit: _Unit):
        torch = self.torch
        stream = unit.stream
        pr, khat, pol, R = self._problem(unit)
        unit.R = R
        unit.plan = self._make_plan(unit, pr, stream)
        with torch.cuda.stream(stream):
            unit.v = torch.zeros((R, unit.plan.n), dtype=torch.complex64, device="cuda")
            unit.x = torch.zeros_like(unit.v)
        ie.ie_rhs_plane_wave(unit.plan.handle, khat, pol, unit.v, stream)
        unit.solver = ie.ie_solver_create(unit.plan.handle, R, self.opts)
        ie.ie_solver_start(unit.solver, unit.v, unit.x, stream)
        ie.ie_solver_advance(unit.solver, 1, stream)       # the first cycle (captures its graph)
        unit.cycles = 1

    def _max_cycles(self) -> int:
        return (self.opts.max_iters + self.opts.restart - 1) // self.opts.restart + 2

    def _state(self, unit: _Unit):
        return ie.ie_solver_state(unit.solver)

    def _advance(self, unit: _Unit):
        ie.ie_solver_advance(unit.solver, 1, unit.stream)
        unit.cycles += 1

    def _engine(self):
        """Advance every live solve by one restart cycle whenever its last one finished."""
        if self.device is not None:
            self.torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                live = list(self.live)
                if not live and self.closing and not self.queue and self.building == 0:
                    self.reap.append(None)
                    self.cv.notify_all()
                    return
            moved = False
            for u in live:
                try:
                    state, info = self._state(u)
                    if state == ie.IE_SOLVER_BUSY:
                        continue
                    if state == ie.IE_SOLVER_IDLE and u.cycles < self._max_cycles():
                        self._advance(u)
                        moved = True
                        continue
                    u.status = ie.IE_OK if info.get("converged") else ie.IE_ERR_NOT_CONVERGED
                    u.info = info
                except Exception as e:
                    u.error = f"{type(e).__name__}: {e}"
                    u.status = -1
                with self.cv:
                    self.live.remove(u)
                    self.reap.append(u)
                    self.cv.notify_all()
                moved = True
            if not moved:
                with self.cv:
                    self.cv.wait(0.0005)

    def _reaper(self):
        """Solutions out, solver and plan torn down (these synchronise the device, so
        they stay off the engine thread), memory given back."""
        if self.device is not None:
            self.torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                while not self.reap:
                    self.cv.wait(0.05)
                unit = self.reap.popleft()
            if unit is None:
                return
            try:
                if unit.stream is not None:
                    unit.stream.synchronize()
                self._harvest(unit, unit.status, unit.info)
            except Exception as e:
                unit.error = unit.error or f"{type(e).__name__}: {e}"
            self._teardown(unit)
            self._complete(unit)

    def _teardown(self, unit: _Unit):
        if unit.solver:
            ie.ie_solver_destroy(unit.solver)
            unit.solver = 0
        unit.v = unit.x = None
        if unit.plan is not None:
            unit.plan.close()
            unit.plan = None


def percentiles(lat, qs=(50, 99)) -> dict:
    a = np.asarray(lat, dtype=np.float64)
    return {f"p{q}": float(np.percentile(a, q)) for q in qs} if a.size else {f"p{q}": None for q in qs}
