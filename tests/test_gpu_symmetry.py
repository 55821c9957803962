"""Symmetry-compressed coupling store (one block per sorted |d|, inputs copied under
the 48 signed axis permutations, output map in the epilogue) against the FP64
oracle, and against the full store."""
import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import dev, empty, host, rel_l2
from test_gpu_parity import ragged_problem

pytestmark = pytest.mark.gpu
BOUND = {ie.IE_PREC_FP32: 1e-6, ie.IE_PREC_BF16X3: 5e-5, ie.IE_PREC_FP16X3: 2e-6, ie.IE_PREC_BF16X1: 1e-2,
         ie.IE_PREC_FP16X1: 2e-3}
ALL = list(BOUND)


def _name(p):
    return ie.PREC_NAMES[p]


def _plan(p, precs=ALL, max_rhs=1, symmetry=1):
    return ie.Plan(ie.problem_from(p, ie.precmask(*precs), max_rhs, symmetry=symmetry))


@pytest.fixture(scope="module")
def tiny():
    p = W.tiny()
    p.alpha = W.alpha_for("tiny")
    return p


def test_canonical_block_counts(tiny):
    """The fully occupied 4^3 grid has 316 far displacements and 16 distinct
    matrices (§2.2); the 16^3 shell has 16,540 groups on 473 blocks."""
    with _plan(tiny, [ie.IE_PREC_FP32]) as plan:
        assert (plan.stats["n_far_disp"], plan.stats["n_coupling_blocks"]) == (316, 16)
    with _plan(W.shell16(), [ie.IE_PREC_FP32]) as plan:
        assert (plan.stats["n_far_disp"], plan.stats["n_coupling_blocks"]) == (16540, 473)


@pytest.mark.parametrize("prec", ALL, ids=_name)
def test_symmetric_full_matvec_tiny(prec, tiny):
    c = W.coefficients(tiny, 2, 701)
    ref = oracle.operator(tiny, c, "full")
    with _plan(tiny, max_rhs=2) as plan:
        y = empty((2, tiny.n))
        ie.ie_matvec(plan.handle, ie.IE_FULL, prec, dev(c), y, 2)
        assert rel_l2(host(y), ref) <= BOUND[prec]


@pytest.mark.parametrize("prec", ALL, ids=_name)
def test_symmetric_translate_ragged(prec):
    p, c = ragged_problem(seed=702, nrhs=3)
    Xr = oracle.aggregate(p, c)
    Yr = oracle.dipole_field(p, Xr, oracle.FAR)
    with _plan(p, max_rhs=3) as plan:
        Y = empty(Xr.shape)
        ie.ie_translate(plan.handle, prec, dev(Xr), Y, 3)
        got = host(Y)
        for r in range(3):
            assert rel_l2(got[r], Yr[r]) <= BOUND[prec], r


def test_symmetric_equals_full_store_shell16():
    """The two stores multiply by the same numbers; the products differ only in FP32 summation
    order (which groups share a partial-sum slab, the order the reductions land), so they agree
    within each one's own rounding error against the oracle: 1e-6 (FP32), 2e-6 (FP16X3)."""
    p = W.shell16()
    c = dev(W.coefficients(p, 1, W.SEED_C["shell16"]))
    out = {}
    for sym in (0, 1):
        with _plan(p, [ie.IE_PREC_FP32, ie.IE_PREC_FP16X3], symmetry=sym) as plan:
            for prec in (ie.IE_PREC_FP32, ie.IE_PREC_FP16X3):
                y = empty((1, p.n))
                ie.ie_matvec(plan.handle, ie.IE_FAR, prec, c, y, 1)
                out[sym, prec] = host(y)
    assert rel_l2(out[1, ie.IE_PREC_FP32], out[0, ie.IE_PREC_FP32]) <= 1e-6
    assert rel_l2(out[1, ie.IE_PREC_FP16X3], out[0, ie.IE_PREC_FP16X3]) <= 2e-6


def test_symmetric_shell16_sampled_and_solve():
    p = W.shell16()
    p.alpha = W.alpha_for("shell16")
    c = W.coefficients(p, 1, W.SEED_C["shell16"])
    targets = W.subsample_boxes(p, 12, W.SEED_SUBSAMPLE["shell16"])
    rows = oracle.basis_rows(p, targets)
    ref = oracle.far_matvec(p, c, targets=targets)
    kh, pol = W.plane_wave_spec(1)
    with _plan(p, [ie.IE_PREC_FP32, ie.IE_PREC_FP16X3]) as plan:
        for prec in (ie.IE_PREC_FP32, ie.IE_PREC_FP16X3):
            y = empty((1, p.n))
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, dev(c), y, 1)
            assert rel_l2(host(y)[:, rows], ref) <= BOUND[prec], _name(prec)
        v = empty((1, p.n))
        ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
        x = empty((1, p.n))
        st, info = ie.ie_solve(plan.handle, v, x, 1, ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X3))
        assert st == ie.IE_OK, info
        xs = host(x)
    vref = oracle.plane_wave_rhs(p, kh, pol)
    Zx = oracle.operator(p, xs, "full", targets=targets)
    res = np.linalg.norm(Zx - vref[:, rows]) / np.linalg.norm(vref[:, rows])
    assert res <= 1e-5, res


def test_symmetric_batch_far_matvec():
    b = W.small_batch()
    R = b.max_rhs
    members = [W.coefficients(m, R, 500 + g) for g, m in enumerate(b.members)]
    refs = [oracle.far_matvec(m, c) for m, c in zip(b.members, members)]
    with ie.Plan(ie.problem_from_batch(b, ie.precmask(ie.IE_PREC_FP32, ie.IE_PREC_FP16X3), symmetry=1)) as plan:
        for prec in (ie.IE_PREC_FP32, ie.IE_PREC_FP16X3):
            y = empty((R, b.n))
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, dev(np.concatenate(members, axis=1)), y, R)
            for g, got in enumerate(b.split(host(y))):
                assert rel_l2(got, refs[g]) <= BOUND[prec], (g, _name(prec))


def test_noalloc_refuses_a_symmetric_plan(tiny):
    with _plan(tiny, [ie.IE_PREC_FP32]) as plan:
        X = empty((1, tiny.n_boxes * 192))
        with pytest.raises(ie.IEError) as e:
            ie.ie_translate_noalloc(plan.handle, X, empty((1, tiny.n_boxes * 192)), 1)
        assert e.value.status == ie.IE_ERR_UNSUPPORTED
