"""ie_translate_noalloc: the FP32 translation that allocates no device memory.

It exists for callers that cannot allocate at call time (device memory owned by
another allocator's pool, or latency-critical loops where cudaMalloc could block);
it must give ie_translate's result.  The check runs two calls in a row, because the
fixed scratch area keeps the previous call's partial sums and must be cleared by
each call.  This file is collected last so that a stop-at-first-failure run has
already run every other test.
"""
import numpy as np
import pytest

import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import dev, empty, host, plan_for, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-6      # the plain FP32 path's tolerance


def _dipole_moments(p, nrhs, seed):
    return W.complex_normal(W.rng(seed), (nrhs, p.n_boxes, 192))


@pytest.mark.parametrize("case", ["tiny", "shell16"])
def test_noalloc_translate_matches_translate_twice(case):
    p = W.tiny() if case == "tiny" else W.shell16()
    nrhs = 2
    X = dev(_dipole_moments(p, nrhs, 300))
    with plan_for(p, max_rhs=nrhs) as plan:
        ref = empty((nrhs, p.n_boxes, 192))
        ie.ie_translate(plan.handle, ie.IE_PREC_FP32, X, ref, nrhs)
        yref = host(ref)
        for _ in range(2):
            out = empty((nrhs, p.n_boxes, 192))
            ie.ie_translate_noalloc(plan.handle, X, out, nrhs)
            assert rel_l2(host(out), yref) <= TOL


def test_noalloc_rejects_requests_beyond_the_fixed_area():
    p = W.tiny()
    with plan_for(p, max_rhs=64) as plan:
        X = empty((64, p.n_boxes, 192))
        Y = empty((64, p.n_boxes, 192))
        with pytest.raises(ie.IEError) as e:
            ie.ie_translate_noalloc(plan.handle, X, Y, 64)
        assert e.value.status == ie.IE_ERR_INVALID
        assert "scratch" in str(e.value)
