"""GPU parity of batched plans: independent scatterers (ragged geometry, ragged nb,
ragged right-hand-side counts) in one plan, each kernel one launch over all of
them, against the FP64 oracle run on each scatterer alone."""
import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import dev, empty, host, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-6
BOUND = {ie.IE_PREC_FP32: TOL, ie.IE_PREC_BF16X3: 5e-5, ie.IE_PREC_FP16X3: 2e-6, ie.IE_PREC_BF16X1: 1e-2,
         ie.IE_PREC_FP16X1: 2e-3}
ALL = list(BOUND)


def _name(p):
    return ie.PREC_NAMES[p]


@pytest.fixture(scope="module")
def batch():
    return W.small_batch()


@pytest.fixture(scope="module")
def coeffs(batch):
    R = batch.max_rhs
    members = [W.coefficients(m, R, 500 + g) for g, m in enumerate(batch.members)]
    return members, np.concatenate(members, axis=1)


@pytest.fixture(scope="module")
def refs(batch, coeffs):
    members, _ = coeffs
    far = [oracle.far_matvec(m, c) for m, c in zip(batch.members, members)]
    near = [oracle.operator(m, c, "near") for m, c in zip(batch.members, members)]
    return dict(far=far, near=near, full=[a + b for a, b in zip(far, near)])


@pytest.fixture(scope="module")
def plan(batch):
    with ie.Plan(ie.problem_from_batch(batch, ie.precmask(*ALL))) as pl:
        yield pl


def test_batch_plan_counts(batch, plan):
    """Far pairs of the batch = the sum over members (no cross-scatterer pair)."""
    total = 0
    for m in batch.members:
        fp = ie.ie_plan_footprint(ie.problem_from(m, ie.precmask(ie.IE_PREC_FP32)))
        assert fp > 0
        d = m.box_ijk[:, None, :].astype(np.int64) - m.box_ijk[None, :, :]
        total += int((np.abs(d).max(axis=2) >= 2).sum())
    assert plan.stats["n_far_pairs"] == total
    assert plan.n == batch.n


@pytest.mark.parametrize("prec", ALL, ids=_name)
def test_batch_far_matvec(prec, batch, coeffs, refs, plan):
    _, packed = coeffs
    R = batch.max_rhs
    y = empty((R, batch.n))
    ie.ie_matvec(plan.handle, ie.IE_FAR, prec, dev(packed), y, R)
    for g, got in enumerate(batch.split(host(y))):
        assert rel_l2(got, refs["far"][g]) <= BOUND[prec], (g, _name(prec))


def test_batch_near_and_full_fp32(batch, coeffs, refs, plan):
    _, packed = coeffs
    R = batch.max_rhs
    for which, key in ((ie.IE_NEAR, "near"), (ie.IE_FULL, "full")):
        y = empty((R, batch.n))
        ie.ie_matvec(plan.handle, which, ie.IE_PREC_FP32, dev(packed), y, R)
        for g, got in enumerate(batch.split(host(y))):
            assert rel_l2(got, refs[key][g]) <= TOL, (g, key)


def test_batch_member_alone_equals_batched(batch, coeffs, plan):
    """A scatterer's product is the same alone and inside the batch."""
    members, packed = coeffs
    R = batch.max_rhs
    y = empty((R, batch.n))
    ie.ie_matvec(plan.handle, ie.IE_FULL, ie.IE_PREC_FP32, dev(packed), y, R)
    inside = batch.split(host(y))
    for g in (0, batch.n_groups - 1):
        m = batch.members[g]
        with ie.Plan(ie.problem_from(m, ie.precmask(ie.IE_PREC_FP32), R)) as alone:
            ya = empty((R, m.n))
            ie.ie_matvec(alone.handle, ie.IE_FULL, ie.IE_PREC_FP32, dev(members[g]), ya, R)
            assert rel_l2(inside[g], host(ya)) <= 5e-7, g   # same terms, other FP32 summation order


def test_batch_plane_waves(batch, plan):
    kh, pol = batch.padded_waves()
    R = batch.max_rhs
    v = empty((R, batch.n))
    ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
    for g, got in enumerate(batch.split(host(v))):
        q = batch.nrhs[g]
        ref = oracle.plane_wave_rhs(batch.members[g], batch.khat[g], batch.pol[g])
        assert rel_l2(got[:q], ref) <= TOL, g
        assert not np.any(got[q:]), g


def _true_residuals(batch, v, x):
    out = []
    for g, (vg, xg) in enumerate(zip(batch.split(v), batch.split(x))):
        q = batch.nrhs[g]
        Zx = oracle.operator(batch.members[g], xg[:q], "full")
        for r in range(q):
            out.append(np.linalg.norm(Zx[r] - vg[r]) / np.linalg.norm(vg[r]))
        assert not np.any(xg[q:]), g          # zero right-hand sides give zero solutions
    return np.array(out)


def test_batch_plain_solve(batch, plan):
    kh, pol = batch.padded_waves()
    R = batch.max_rhs
    v = empty((R, batch.n))
    ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
    x = empty((R, batch.n))
    st, info = ie.ie_solve(plan.handle, v, x, R, ie.solve_opts(tol=1e-6, restart=50))
    assert st == ie.IE_OK, info
    res = _true_residuals(batch, host(v), host(x))
    assert res.max() <= 2e-6, res


def test_batch_mixed_solve(batch, plan):
    kh, pol = batch.padded_waves()
    R = batch.max_rhs
    v = empty((R, batch.n))
    ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
    x = empty((R, batch.n))
    st, info = ie.ie_solve(plan.handle, v, x, R,
                           ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_BF16X3, refine=1,
                                         refine_prec=ie.IE_PREC_FP16X3, inner_tol=1e-3))
    assert st == ie.IE_OK, info
    res = _true_residuals(batch, host(v), host(x))
    assert res.max() <= 1e-5, res


def test_batch_solve_member_alone_same_iterations(batch, plan):
    """Systems of one batch run their own GMRES: a member solved alone takes the
    iterations it takes inside the batch (the batch reports the maximum)."""
    kh, pol = batch.padded_waves()
    R = batch.max_rhs
    its = []
    for g, m in enumerate(batch.members):
        with ie.Plan(ie.problem_from(m, ie.precmask(ie.IE_PREC_FP32), R)) as alone:
            v = empty((R, m.n))
            ie.ie_rhs_plane_wave(alone.handle, kh[g], pol[g], v)
            x = empty((R, m.n))
            st, info = ie.ie_solve(alone.handle, v, x, R, ie.solve_opts(tol=1e-6, restart=50))
            assert st == ie.IE_OK
            its.append(info["iterations"])
    v = empty((R, batch.n))
    ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
    x = empty((R, batch.n))
    st, info = ie.ie_solve(plan.handle, v, x, R, ie.solve_opts(tol=1e-6, restart=50))
    assert st == ie.IE_OK
    assert abs(info["iterations"] - max(its)) <= 1, (info, its)   # rounding may move the last step


@pytest.fixture(scope="module")
def plan_exact(batch):
    with ie.Plan(ie.problem_from_batch(batch, ie.precmask(ie.IE_PREC_FP32, ie.IE_PREC_FP16X3), exact_rhs=True)) as pl:
        yield pl


@pytest.mark.parametrize("prec", [ie.IE_PREC_FP32, ie.IE_PREC_FP16X3], ids=_name)
def test_batch_exact_rhs_far_matvec(prec, batch, coeffs, refs, plan_exact):
    """With per-scatterer right-hand-side counts, a member's own columns match the
    oracle and its padding columns get no far-zone contribution."""
    _, packed = coeffs
    R = batch.max_rhs
    y = empty((R, batch.n))
    ie.ie_matvec(plan_exact.handle, ie.IE_FAR, prec, dev(packed), y, R)
    for g, got in enumerate(batch.split(host(y))):
        q = batch.nrhs[g]
        assert rel_l2(got[:q], refs["far"][g][:q]) <= BOUND[prec], (g, _name(prec))
        assert not np.any(got[q:]), g


def test_batch_exact_rhs_solve(batch, plan_exact):
    kh, pol = batch.padded_waves()
    R = batch.max_rhs
    v = empty((R, batch.n))
    ie.ie_rhs_plane_wave(plan_exact.handle, kh, pol, v)
    x = empty((R, batch.n))
    st, info = ie.ie_solve(plan_exact.handle, v, x, R, ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X3))
    assert st == ie.IE_OK, info
    res = _true_residuals(batch, host(v), host(x))
    assert res.max() <= 1e-5, res
