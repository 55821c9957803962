"""Continuous serving of scattering solves on one GPU over the C ABI.

Requests (one scatterer, 1-4 plane-wave excitations each) arrive over time.  The
scheduler admits them in arrival order while their device footprint
(ie_plan_footprint + ie_solver_footprint, plus the request's vectors) fits the
HBM budget; an admitted request runs on its own worker thread and CUDA stream:
plan (coupling and near blocks), excitation, GMRES (optionally with FP64
refinement), teardown.  With `batch` > 1 the requests queued behind the head
that share its grid are merged into one batched plan (independent scatterers in
one plan, one launch per kernel) and solved together.  Every device step runs in
libie; this module only orders the calls.
"""
from __future__ import annotations

import collections
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


class Server:
    """FIFO admission by device footprint; one worker thread per admitted unit of work.

    precs / opts: the plan's precisions and the ie_solve options of every request.
    budget: device bytes the server may hold at once.  batch: most requests merged
    into one plan (same grid only).  keep_solutions: keep each request's solution.
    symmetry: 1 builds symmetry-compressed plans (one coupling block per sorted |d|).
    """

    def __init__(self, precs, opts, budget: int, workers: int = 4, batch: int = 1, keep_solutions: bool = False,
                 symmetry: int = 0):
        import torch
        self.torch = torch
        self.mask = ie.precmask(*precs)
        self.opts = opts
        self.budget = int(budget)
        self.batch = max(1, int(batch))
        self.keep = keep_solutions
        self.symmetry = int(symmetry)
        self.queue: collections.deque = collections.deque()
        self.done: list = []
        self.used = 0
        self.cv = threading.Condition()
        self.closing = False
        self.t0 = time.perf_counter()
        self.peak_used = 0
        self.workers = [threading.Thread(target=self._worker, daemon=True) for _ in range(workers)]
        self.device = torch.cuda.current_device() if torch.cuda.is_available() else None
        for w in self.workers:
            w.start()

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
        for w in self.workers:
            w.join()

    # ---------------------------------------------------------------- scheduler
    def footprint_of(self, req: Request, R: int = 4) -> int:
        """Device bytes of `req` in a plan of R columns (R >= its own nrhs): the plan
        (ie_plan_footprint), the inner GMRES state, the refinement vectors and v, x.
        Members of a merged plan share its coupling store, so a batch needs at most
        the sum of its members' footprints at the batch's column count."""
        R = max(R, req.nrhs)
        n = int(req.problem.nb.sum())
        plan_b = ie.ie_plan_footprint(ie.problem_from(req.problem, self.mask, R, symmetry=self.symmetry))
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
            if self.used + need <= self.budget or (self.used == 0 and len(group) == 1):
                for r in group:
                    self.queue.remove(r)
                return group, need
            if len(group) == 1:
                return None, 0          # head-of-line waits for memory
            group.pop()
        return None, 0

    def _worker(self):
        torch = self.torch
        stream = None
        if self.device is not None:
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream()
        while True:
            with self.cv:
                while True:
                    if self.closing and not self.queue:
                        return
                    group, need = self._take()
                    if group:
                        self.used += need
                        self.peak_used = max(self.peak_used, self.used)
                        break
                    self.cv.wait(0.05)
            t_start = self.now()
            try:
                self._run(group, stream)
            except Exception as e:   # the request fails; the server keeps serving
                for r in group:
                    r.error = f"{type(e).__name__}: {e}"
            t_done = self.now()
            with self.cv:
                self.used -= need
                for r in group:
                    r.t_start, r.t_done = t_start, t_done
                    self.done.append(r)
                self.cv.notify_all()

    def _run(self, group, stream):
        torch = self.torch
        with torch.cuda.stream(stream):
            if len(group) == 1:
                r = group[0]
                pr = ie.problem_from(r.problem, self.mask, r.nrhs, symmetry=self.symmetry)
                khat, pol, R = r.khat, r.pol, r.nrhs
            else:
                view = _BatchView(group)
                pr = ie.problem_from_batch(view, self.mask, symmetry=self.symmetry, exact_rhs=True)
                R = view.R
                khat = np.zeros((len(group), R, 3))
                khat[:, :, 2] = 1.0
                pol = np.zeros((len(group), R, 3))
                for g, r in enumerate(group):
                    khat[g, :r.nrhs] = np.asarray(r.khat).reshape(-1, 3)
                    pol[g, :r.nrhs] = np.asarray(r.pol).reshape(-1, 3)
            plan = ie.Plan(pr, stream)
            try:
                n = plan.n
                v = torch.zeros((R, n), dtype=torch.complex64, device="cuda")
                x = torch.zeros_like(v)
                ie.ie_rhs_plane_wave(plan.handle, khat, pol, v, stream)
                st, info = ie.ie_solve(plan.handle, v, x, R, self.opts, stream)
                stream.synchronize()
                off = 0
                for r in group:
                    nr = int(r.problem.nb.sum())
                    r.status, r.info = st, dict(info)
                    if self.keep:
                        r.x = x[:r.nrhs, off:off + nr].clone()
                    off += nr
                del v, x
            finally:
                plan.close()


def percentiles(lat, qs=(50, 99)) -> dict:
    a = np.asarray(lat, dtype=np.float64)
    return {f"p{q}": float(np.percentile(a, q)) for q in qs} if a.size else {f"p{q}": None for q in qs}
