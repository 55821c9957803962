"""GPU parity of the tcgen05 translation and the mixed-precision solve against the
FP64 oracle, through the C ABI.

Stated bounds (relative L2), from the split arithmetic: bf16 hi + lo keeps ~16
significant bits and the dropped lo*lo term is ~2^-16 of each product, so BF16X3
<= 5e-5; fp16 hi + lo keeps ~22 bits, FP16X3 <= 2e-6; one bf16 product (8 bits)
BF16X1 <= 1e-2; one fp16 product (11 bits, 2^3 finer) FP16X1 <= 2e-3.  The mixed solve (inner GMRES on BF16X3 products, FP64 refinement
residual from FP32 products) must reach a true residual <= 1e-5.
"""
import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import box_errors, dev, empty, host, plan_for, rel_l2
from test_gpu_parity import ragged_problem

pytestmark = pytest.mark.gpu
BOUND = {ie.IE_PREC_BF16X3: 5e-5, ie.IE_PREC_FP16X3: 2e-6, ie.IE_PREC_BF16X1: 1e-2, ie.IE_PREC_FP16X1: 2e-3}
TC = [ie.IE_PREC_BF16X3, ie.IE_PREC_FP16X3, ie.IE_PREC_BF16X1, ie.IE_PREC_FP16X1]
ALL = [ie.IE_PREC_FP32] + TC


def _name(p):
    return ie.PREC_NAMES[p]


@pytest.fixture(scope="module")
def tiny():
    p = W.tiny()
    p.alpha = W.alpha_for("tiny")
    return p


@pytest.mark.parametrize("prec", TC, ids=_name)
def test_tc_translate_tiny(prec, tiny):
    Xr = oracle.aggregate(tiny, W.coefficients(tiny, 1, 400))
    Yr = oracle.dipole_field(tiny, Xr, oracle.FAR)
    with plan_for(tiny, precs=ALL) as plan:
        Y = empty(Xr.shape)
        ie.ie_translate(plan.handle, prec, dev(Xr), Y, 1)
        assert rel_l2(host(Y), Yr) <= BOUND[prec]


@pytest.mark.parametrize("prec", TC, ids=_name)
def test_tc_translate_ragged_multi_rhs(prec):
    p, c = ragged_problem(seed=410, nrhs=3)
    Xr = oracle.aggregate(p, c)
    Yr = oracle.dipole_field(p, Xr, oracle.FAR)
    with plan_for(p, precs=ALL, max_rhs=3) as plan:
        Y = empty(Xr.shape)
        ie.ie_translate(plan.handle, prec, dev(Xr), Y, 3)
        got = host(Y)
        for r in range(3):
            assert rel_l2(got[r], Yr[r]) <= BOUND[prec]


@pytest.mark.parametrize("prec", TC, ids=_name)
def test_tc_full_matvec_tiny(prec, tiny):
    c = W.coefficients(tiny, 2, 401)
    ref = oracle.operator(tiny, c, "full")
    with plan_for(tiny, precs=ALL, max_rhs=2) as plan:
        y = empty((2, tiny.n))
        ie.ie_matvec(plan.handle, ie.IE_FULL, prec, dev(c), y, 2)
        assert rel_l2(host(y), ref) <= BOUND[prec]


def test_tc_degenerate_and_large_dynamic_range():
    """One far pair each way, and P scaled by 2^20 (fp16 needs its per-block scaling)."""
    g = W.rng(402)
    ijk = np.array([(0, 0, 0), (2, 0, 0), (0, 7, 1)], dtype=np.int32)
    nb = np.array([1, 192, 40], dtype=np.int32)
    P = W.random_P(g, nb) * 2.0 ** 20
    p = W.Problem(name="deg", G=10, box_ijk=ijk, nb=nb, P=P, alpha=1.0)
    c = W.coefficients(p, 1, 403)
    ref = oracle.far_matvec(p, c)
    with plan_for(p, precs=ALL) as plan:
        for prec in TC:
            y = empty((1, p.n))
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, dev(c), y, 1)
            assert rel_l2(host(y), ref) <= BOUND[prec], _name(prec)


@pytest.mark.parametrize("prec", [ie.IE_PREC_BF16X3, ie.IE_PREC_FP16X3], ids=_name)
def test_tc_full_size_shell16_sampled(prec):
    p = W.shell16()
    c = W.coefficients(p, 1, W.SEED_C["shell16"])
    targets = W.subsample_boxes(p, 12, W.SEED_SUBSAMPLE["shell16"])
    with plan_for(p, precs=[ie.IE_PREC_FP32, prec]) as plan:
        y = empty((1, p.n))
        ie.ie_matvec(plan.handle, ie.IE_FAR, prec, dev(c), y, 1)
        got = host(y)[:, oracle.basis_rows(p, targets)]
    ref = oracle.far_matvec(p, c, targets=targets)
    assert rel_l2(got, ref) <= BOUND[prec]
    # every sampled box on its own (10x: the spread of per-box cancellation; a fault in one
    # box or displacement class would give O(1) there)
    worst = box_errors(got, ref, np.asarray(p.nb)[targets]).max()
    assert worst <= 10 * BOUND[prec], worst


@pytest.mark.parametrize("inner", [ie.IE_PREC_BF16X3, ie.IE_PREC_BF16X1, ie.IE_PREC_FP16X1], ids=_name)
def test_mixed_solve_with_refinement_tiny(inner, tiny):
    Z = oracle.dense_operator(tiny)
    kh, pol = W.plane_wave_spec(2, seed=404)
    v = oracle.plane_wave_rhs(tiny, kh, pol)
    with plan_for(tiny, precs=ALL, max_rhs=2) as plan:
        x = empty((2, tiny.n))
        st, info = ie.ie_solve(plan.handle, dev(v), x, 2,
                               ie.solve_opts(tol=1e-5, prec=inner, refine=1, refine_prec=ie.IE_PREC_FP32,
                                             inner_tol=1e-2 if inner == ie.IE_PREC_BF16X1 else 1e-3))
        assert st == ie.IE_OK, info
        xs = host(x)
    for r in range(2):
        res = np.linalg.norm(v[r] - Z @ xs[r]) / np.linalg.norm(v[r])
        assert res <= 1e-5, (r, res)


def test_mixed_solve_shell16_true_residual():
    p = W.shell16()
    p.alpha = W.alpha_for("shell16")
    kh, pol = W.plane_wave_spec(1)
    targets = W.subsample_boxes(p, 12, W.SEED_SUBSAMPLE["shell16"])
    with plan_for(p, precs=[ie.IE_PREC_FP32, ie.IE_PREC_BF16X3]) as plan:
        v = empty((1, p.n))
        ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
        x = empty((1, p.n))
        st, info = ie.ie_solve(plan.handle, v, x, 1,
                               ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_BF16X3, refine=1,
                                             refine_prec=ie.IE_PREC_FP32, inner_tol=1e-3))
        assert st == ie.IE_OK, info
        xs = host(x)
    vref = oracle.plane_wave_rhs(p, kh, pol)
    rows = oracle.basis_rows(p, targets)
    Zx = oracle.operator(p, xs, "full", targets=targets)
    res = np.linalg.norm(Zx - vref[:, rows]) / np.linalg.norm(vref[:, rows])
    assert res <= 1e-5, res


def test_tc_plan_without_fp32_store():
    """A plan of 16-bit precisions only cuts its images from a staging buffer in
    chunks (shell16: 16,540 displacements, several chunks) and keeps no FP32 store."""
    p = W.shell16()
    c = W.coefficients(p, 1, W.SEED_C["shell16"])
    targets = W.subsample_boxes(p, 12, W.SEED_SUBSAMPLE["shell16"])
    ref = oracle.far_matvec(p, c, targets=targets)
    rows = oracle.basis_rows(p, targets)
    mask16 = ie.precmask(ie.IE_PREC_BF16X3, ie.IE_PREC_FP16X3)
    mask_all = ie.precmask(ie.IE_PREC_FP32, ie.IE_PREC_BF16X3, ie.IE_PREC_FP16X3)
    assert ie.ie_plan_footprint(ie.problem_from(p, mask16)) < ie.ie_plan_footprint(ie.problem_from(p, mask_all))
    with plan_for(p, precs=[ie.IE_PREC_BF16X3, ie.IE_PREC_FP16X3]) as plan:
        for prec in (ie.IE_PREC_BF16X3, ie.IE_PREC_FP16X3):
            y = empty((1, p.n))
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, dev(c), y, 1)
            assert rel_l2(host(y)[:, rows], ref) <= BOUND[prec], _name(prec)
        y = empty((1, p.n))
        with pytest.raises(ie.IEError) as e:
            ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_FP32, dev(c), y, 1)
        assert e.value.status == ie.IE_ERR_UNSUPPORTED
        X = empty((1, p.n_boxes * 192))
        with pytest.raises(ie.IEError) as e:
            ie.ie_translate_noalloc(plan.handle, X, empty((1, p.n_boxes * 192)), 1)
        assert e.value.status == ie.IE_ERR_UNSUPPORTED


def test_mixed_solve_one_fp16_store_shell16():
    """Inner GMRES on FP16X1 products, refinement residual from FP16X3: one store."""
    p = W.shell16()
    p.alpha = W.alpha_for("shell16")
    kh, pol = W.plane_wave_spec(1)
    targets = W.subsample_boxes(p, 12, W.SEED_SUBSAMPLE["shell16"])
    with plan_for(p, precs=[ie.IE_PREC_FP16X1, ie.IE_PREC_FP16X3]) as plan:
        v = empty((1, p.n))
        ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
        x = empty((1, p.n))
        st, info = ie.ie_solve(plan.handle, v, x, 1,
                               ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X1, refine=1,
                                             refine_prec=ie.IE_PREC_FP16X3, inner_tol=1e-3))
        assert st == ie.IE_OK, info
        xs = host(x)
    vref = oracle.plane_wave_rhs(p, kh, pol)
    rows = oracle.basis_rows(p, targets)
    Zx = oracle.operator(p, xs, "full", targets=targets)
    res = np.linalg.norm(Zx - vref[:, rows]) / np.linalg.norm(vref[:, rows])
    assert res <= 1e-5, res


def test_fp16x3_solve_shell16_true_residual():
    """GMRES(50) directly on FP16X3 products to 1e-5, no refinement: the true residual
    against the FP64 operator stays within 1e-5."""
    p = W.shell16()
    p.alpha = W.alpha_for("shell16")
    kh, pol = W.plane_wave_spec(1)
    targets = W.subsample_boxes(p, 12, W.SEED_SUBSAMPLE["shell16"])
    with plan_for(p, precs=[ie.IE_PREC_FP16X3]) as plan:
        v = empty((1, p.n))
        ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
        x = empty((1, p.n))
        st, info = ie.ie_solve(plan.handle, v, x, 1, ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X3))
        assert st == ie.IE_OK, info
        xs = host(x)
    vref = oracle.plane_wave_rhs(p, kh, pol)
    rows = oracle.basis_rows(p, targets)
    Zx = oracle.operator(p, xs, "full", targets=targets)
    res = np.linalg.norm(Zx - vref[:, rows]) / np.linalg.norm(vref[:, rows])
    assert res <= 1e-5, res


def test_autotuner_choice_is_valid_and_products_stay_correct():
    """ie_plan_tune times 8 configurations, keeps the fastest, and the plan's products
    with the tuned work lists still match the oracle."""
    p, c = ragged_problem(seed=430, nrhs=3)
    ref = oracle.operator(p, c, "full")
    with plan_for(p, precs=ALL, max_rhs=3) as plan:
        for prec in (ie.IE_PREC_FP16X3, ie.IE_PREC_BF16X1):
            info = ie.ie_plan_tune(plan.handle, prec, 3)
            assert info["tile_columns"] in (96, 80, 64, 48) and info["order"] in (0, 1), info
            assert info["candidates"] == 8 and 0 < info["ms"] <= info["default_ms"], info
            y = empty((3, p.n))
            ie.ie_matvec(plan.handle, ie.IE_FULL, prec, dev(c), y, 3)
            assert rel_l2(host(y), ref) <= BOUND[prec], _name(prec)
        with pytest.raises(ie.IEError):
            ie.ie_plan_tune(plan.handle, ie.IE_PREC_FP32, 1)


def test_translation_abort_path_reports_timeout_and_recovers(tiny):
    """A real tensor-core launch driven through its abort path: with the pipeline's waits
    limited to 64 SM cycles the roles give up at once; the drains (default limit) still
    wait for the copies and MMAs in flight, TMEM is freed, the plan reports IE_ERR_TIMEOUT,
    and with the default limit back the next product on the same plan is correct."""
    c = W.coefficients(tiny, 1, 211)
    ref = oracle.far_matvec(tiny, c)
    with plan_for(tiny, precs=[ie.IE_PREC_FP16X3]) as plan:
        y = empty((1, tiny.n))
        try:
            ie.ie_diag_wait_limit(64)
            ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_FP16X3, dev(c), y, 1)
            with pytest.raises(ie.IEError) as e:
                ie.ie_plan_check(plan.handle)
            assert e.value.status == ie.IE_ERR_TIMEOUT
        finally:
            ie.ie_diag_wait_limit(0)
        ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_FP16X3, dev(c), y, 1)
        assert ie.ie_plan_check(plan.handle) == ie.IE_OK
        assert rel_l2(host(y), ref) <= BOUND[ie.IE_PREC_FP16X3]
