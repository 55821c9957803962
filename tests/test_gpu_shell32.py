"""Full-size shell32 (32^3 grid, radius-14 sphere shell: 5,000 boxes, 160,000 basis
unknowns, 24.9 M far pairs in 112,160 displacement groups): every product form on a
seeded 64-box target subsample against the FP64 oracle, and the mixed solve's true
residual on the same subsample (the FP64 refinement reports the full residual).

Per-box errors: beside the vector-wide relative error, every sampled box's own relative
error must stay within PER_BOX x the precision's bound.  The bounds hold per product
term, so a box's error exceeds the vector's only by how much its field cancels (the
ratio of sum |G||x| to |sum G x| over its sources), a few units on these shells; a fault
in one displacement class or box gives O(1) errors there."""
import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import box_errors, dev, empty, host, rel_l2

pytestmark = pytest.mark.gpu
BOUND = {ie.IE_PREC_FP32: 1e-6, ie.IE_PREC_BF16X3: 5e-5, ie.IE_PREC_FP16X3: 2e-6, ie.IE_PREC_FP16X1: 2e-3}
PER_BOX = 10


@pytest.fixture(scope="module")
def p():
    p = W.shell32()
    p.alpha = W.alpha_for("shell32")
    return p


@pytest.fixture(scope="module")
def targets(p):
    return W.subsample_boxes(p, 64, W.SEED_SUBSAMPLE["shell32"])


@pytest.fixture(scope="module")
def plan(p):
    with ie.Plan(ie.problem_from(p, ie.precmask(*BOUND))) as pl:
        yield pl


def test_shell32_plan_counts(p, plan):
    st = plan.stats
    assert (st["n_boxes"], st["n_far_pairs"], st["n_far_disp"]) == (5000, 24910952, 112160)
    assert st["n"] == p.n == 160000


def test_shell32_far_products_sampled(p, targets, plan):
    c = W.coefficients(p, 1, W.SEED_C["shell32"])
    ref = oracle.far_matvec(p, c, targets=targets)
    rows = oracle.basis_rows(p, targets)
    cd = dev(c)
    for prec, bound in BOUND.items():
        y = empty((1, p.n))
        ie.ie_matvec(plan.handle, ie.IE_FAR, prec, cd, y, 1)
        got = host(y)[:, rows]
        err = rel_l2(got, ref)
        worst = box_errors(got, ref, np.asarray(p.nb)[targets]).max()
        assert err <= bound and worst <= PER_BOX * bound, (ie.PREC_NAMES[prec], err, worst)


SOLVES = {
    "bf16x3_refined": dict(tol=1e-5, prec=ie.IE_PREC_BF16X3, refine=1, refine_prec=ie.IE_PREC_FP16X3, inner_tol=1e-3),
    "fp16x3": dict(tol=1e-5, prec=ie.IE_PREC_FP16X3),
}


@pytest.mark.parametrize("form", list(SOLVES))
def test_shell32_mixed_solve_residual(form, p, targets, plan):
    kh, pol = W.plane_wave_spec(1)
    v = empty((1, p.n))
    ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
    x = empty((1, p.n))
    st, info = ie.ie_solve(plan.handle, v, x, 1, ie.solve_opts(**SOLVES[form]))
    assert st == ie.IE_OK and info["relres"] <= 1e-5, info
    xs = host(x)
    vref = oracle.plane_wave_rhs(p, kh, pol)
    rows = oracle.basis_rows(p, targets)
    Zx = oracle.operator(p, xs, "full", targets=targets)
    res = np.linalg.norm(Zx - vref[:, rows]) / np.linalg.norm(vref[:, rows])
    assert res <= 1e-5, res
