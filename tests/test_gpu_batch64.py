"""batch64 at full size (64 scatterers, 165,968 boxes, 735 M far pairs, each scatterer
translating only its own right-hand sides) in the configuration bench.py times:
FP16X3 far products sampled on a few target boxes of four scatterers against the FP64
oracle run on each of them alone."""
import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import dev, empty, host, rel_l2

pytestmark = pytest.mark.gpu


def test_batch64_sampled_far_products():
    b = W.batch64()
    R = b.max_rhs
    members = [W.coefficients(m, R, 500 + g) for g, m in enumerate(b.members)]
    for g, q in enumerate(b.nrhs):
        members[g][q:] = 0          # padding columns carry no right-hand side
    with ie.Plan(ie.problem_from_batch(b, ie.precmask(ie.IE_PREC_FP16X3), exact_rhs=True)) as plan:
        y = empty((R, b.n))
        ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_FP16X3, dev(np.concatenate(members, axis=1)), y, R)
        ie.ie_plan_check(plan.handle)
        got = b.split(host(y))
    sizes = [m.n_boxes for m in b.members]
    picks = sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), 1, 40})
    for g in picks:
        m, q = b.members[g], b.nrhs[g]
        targets = W.subsample_boxes(m, 6, 900 + g)
        rows = oracle.basis_rows(m, targets)
        ref = oracle.far_matvec(m, members[g][:q], targets=targets)
        assert rel_l2(got[g][:q, rows], ref) <= 2e-6, g
        assert not np.any(got[g][q:]), g
