"""ie_translate_noalloc: the FP32 translation that allocates no device memory.

It exists for callers that cannot allocate at call time (device memory owned by
another allocator's pool, or latency-critical loops where cudaMalloc could block);
it must give ie_translate's result.  The check runs two calls in a row, because the
fixed scratch area keeps the previous call's partial sums and must be cleared by
each call.  This file is collected last so that a stop-at-first-failure run has
already run every other test.
"""
import pytest

import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import dev, empty, host, plan_for, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-6      # the plain FP32 path's tolerance
AREA = 32 << 20  # bytes of the library's fixed scratch area
SLABS = 8        # FP32 partial-sum slabs the translation keeps


def _dipole_moments(n_boxes, nrhs, seed):
    return W.complex_normal(W.rng(seed), (nrhs, n_boxes, 192))


def _scratch_need(n_boxes, nrhs):
    return SLABS * nrhs * n_boxes * 192 * 8


def _check_twice(plan, n_boxes, nrhs, seed):
    X = dev(_dipole_moments(n_boxes, nrhs, seed))
    ref = empty((nrhs, n_boxes, 192))
    ie.ie_translate(plan.handle, ie.IE_PREC_FP32, X, ref, nrhs)
    yref = host(ref)
    for _ in range(2):
        out = empty((nrhs, n_boxes, 192))
        ie.ie_translate_noalloc(plan.handle, X, out, nrhs)
        assert rel_l2(host(out), yref) <= TOL


@pytest.mark.parametrize("case", ["tiny", "shell16"])
def test_noalloc_translate_matches_translate_twice(case):
    p = W.tiny() if case == "tiny" else W.shell16()
    nrhs = 2
    # the case must fit the fixed area (shell16 at 2 right-hand sides uses ~29.5 MiB of 32)
    assert _scratch_need(p.n_boxes, nrhs) <= AREA, (case, _scratch_need(p.n_boxes, nrhs))
    with plan_for(p, max_rhs=nrhs) as plan:
        _check_twice(plan, p.n_boxes, nrhs, 300)


def test_noalloc_translate_batched_plan():
    """Several scatterers in one plan (one launch over all their groups), every column
    translated (no per-scatterer right-hand-side counts)."""
    b = W.small_batch()
    nrhs = 2
    pr = ie.problem_from_batch(b, ie.precmask(ie.IE_PREC_FP32), max_rhs=nrhs)
    with ie.Plan(pr) as plan:
        assert plan.stats["n_groups"] == len(b.members) > 1
        _check_twice(plan, plan.stats["n_boxes"], nrhs, 301)


def test_noalloc_translate_replays_from_a_captured_graph():
    """After the first call has set the area up on the device, a call launches kernels
    only (no allocation, no host copy), so it can be captured into a CUDA graph; each
    replay clears the partial sums again and gives ie_translate's result."""
    import torch
    p = W.tiny()
    nrhs = 2
    with plan_for(p, max_rhs=nrhs) as plan:
        X = dev(_dipole_moments(p.n_boxes, nrhs, 302))
        ref = empty((nrhs, p.n_boxes, 192))
        ie.ie_translate(plan.handle, ie.IE_PREC_FP32, X, ref, nrhs)
        yref = host(ref)
        out = empty((nrhs, p.n_boxes, 192))
        ie.ie_translate_noalloc(plan.handle, X, out, nrhs)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ie.ie_translate_noalloc(plan.handle, X, out, nrhs)
        for _ in range(2):
            out.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert rel_l2(host(out), yref) <= TOL


def test_noalloc_rejects_requests_beyond_the_fixed_area():
    p = W.tiny()
    with plan_for(p, max_rhs=64) as plan:
        assert _scratch_need(p.n_boxes, 64) > AREA
        X = empty((64, p.n_boxes, 192))
        Y = empty((64, p.n_boxes, 192))
        with pytest.raises(ie.IEError) as e:
            ie.ie_translate_noalloc(plan.handle, X, Y, 64)
        assert e.value.status == ie.IE_ERR_INVALID
        assert "scratch" in str(e.value)
