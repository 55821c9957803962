"""The serving loop on the GPU: requests admitted by footprint, run alone or merged
into batched plans, each solution checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import host, torch_cuda
from paper_2501_04684_gb300 import serve as S

pytestmark = pytest.mark.gpu


def _requests():
    b = W.small_batch()
    return [S.Request(rid=g, problem=m, khat=b.khat[g], pol=b.pol[g]) for g, m in enumerate(b.members)]


def _serve(batch):
    torch = torch_cuda()
    opts = ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X1, refine=1, refine_prec=ie.IE_PREC_FP16X3, inner_tol=1e-3)
    free, _ = torch.cuda.mem_get_info()
    srv = S.Server([ie.IE_PREC_FP16X1, ie.IE_PREC_FP16X3], opts, int(free * 0.5), workers=2, batch=batch,
                   keep_solutions=True)
    reqs = _requests()
    try:
        for r in reqs:
            srv.submit(r)
        done = srv.drain(len(reqs), timeout=600)
    finally:
        srv.close()
    assert srv.peak_used <= srv.budget
    return {r.rid: r for r in done}


@pytest.mark.parametrize("batch", [1, 4])
def test_served_solutions_meet_tolerance(batch):
    out = _serve(batch)
    for rid, r in sorted(out.items()):
        assert r.status == ie.IE_OK, (rid, r.error, r.info)
        v = oracle.plane_wave_rhs(r.problem, r.khat, r.pol)
        x = host(r.x)
        Zx = oracle.operator(r.problem, x, "full")
        for q in range(r.nrhs):
            res = np.linalg.norm(Zx[q] - v[q]) / np.linalg.norm(v[q])
            assert res <= 1e-5, (rid, q, res)


def test_request_alone_and_in_a_batch_agree():
    alone, merged = _serve(1), _serve(4)
    for rid in alone:
        a, m = host(alone[rid].x), host(merged[rid].x)
        assert np.linalg.norm(a - m) / np.linalg.norm(a) <= 5e-4, rid
