"""The serving loop on the GPU: requests admitted by footprint, their plans attached to a
shared coupling-block store, run alone or merged into batched plans, either stepped one
restart cycle at a time (GMRES on FP16X3 products to 1e-5) or blocking with FP64
refinement (GMRES on FP16X1 products inside); each solution is checked against the FP64
oracle.

Alone against in the mix.  A served solution x_i of Z x = v has the true residual
r_i = v - Z x_i with ||r_i|| <= tol ||v|| (checked against the oracle).  Two of them
differ by Z^-1 (r_2 - r_1), and ||x_1|| >= (1 - tol) ||v|| / ||Z||, so
    ||x_1 - x_2|| / ||x_1|| <= 2 tol kappa(Z) / (1 - tol),
kappa(Z) the condition number of the scatterer's operator, taken here from the SVD of
the oracle's dense Z (the members are small).
"""
import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import host, torch_cuda
from paper_2501_04684_gb300 import serve as S

pytestmark = pytest.mark.gpu
TOL = 1e-5
MODES = {
    "stepped": ([ie.IE_PREC_FP16X3], dict(tol=TOL, prec=ie.IE_PREC_FP16X3)),
    "refined": ([ie.IE_PREC_FP16X1, ie.IE_PREC_FP16X3],
                dict(tol=TOL, prec=ie.IE_PREC_FP16X1, refine=1, refine_prec=ie.IE_PREC_FP16X3, inner_tol=1e-3)),
}


def _requests():
    b = W.small_batch()
    return [S.Request(rid=g, problem=m, khat=b.khat[g], pol=b.pol[g]) for g, m in enumerate(b.members)]


def _serve(batch, mode):
    torch = torch_cuda()
    precs, kw = MODES[mode]
    free, _ = torch.cuda.mem_get_info()
    srv = S.Server(precs, ie.solve_opts(**kw), int(free * 0.5), workers=2, batch=batch, keep_solutions=True,
                   symmetry=1)
    assert srv.share and srv.stepped == (mode == "stepped")
    reqs = _requests()
    try:
        for r in reqs:
            srv.submit(r)
        done = srv.drain(len(reqs), timeout=600)
        n_stores = len(srv.stores)
    finally:
        srv.close()
    assert srv.peak_used <= srv.budget and srv.used == srv.store_bytes
    assert n_stores == 1          # one store for the four scatterers (same k, eta, a)
    return {r.rid: r for r in done}


@pytest.fixture(scope="module")
def kappas():
    """Condition numbers of the members' dense operators (oracle, SVD)."""
    out = {}
    for r in _requests():
        s = np.linalg.svd(oracle.dense_operator(r.problem), compute_uv=False)
        out[r.rid] = float(s[0] / s[-1])
    return out


@pytest.mark.parametrize("mode", ["stepped", "refined"])
@pytest.mark.parametrize("batch", [1, 4])
def test_served_solutions_meet_tolerance(batch, mode):
    out = _serve(batch, mode)
    for rid, r in sorted(out.items()):
        assert r.status == ie.IE_OK, (rid, r.error, r.info)
        v = oracle.plane_wave_rhs(r.problem, r.khat, r.pol)
        x = host(r.x)
        Zx = oracle.operator(r.problem, x, "full")
        for q in range(r.nrhs):
            res = np.linalg.norm(Zx[q] - v[q]) / np.linalg.norm(v[q])
            assert res <= TOL, (rid, q, res)


@pytest.mark.parametrize("mode", ["stepped", "refined"])
def test_request_alone_and_in_a_batch_agree(mode, kappas):
    alone, merged = _serve(1, mode), _serve(4, mode)
    for rid in alone:
        a, m = host(alone[rid].x), host(merged[rid].x)
        bound = 2 * TOL * kappas[rid] / (1 - TOL)
        assert np.linalg.norm(a - m) / np.linalg.norm(a) <= bound, (rid, bound)
